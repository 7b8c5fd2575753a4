"""CPU tests of the C ABI library: it builds, loads, exports every declared symbol, and its
host-only logic (FP64 Pade plan, argument validation) agrees with the oracle.  No compute
call needs a GPU here."""
import math
import os
import re

import numpy as np
import pytest

from oracle import sssp_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2511_03343_gb300 import build
    build.build()
    from paper_2511_03343_gb300 import sssp
    return sssp.lib()


def _declared_symbols():
    syms = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(pe_\w+)\s*\(", txt))
    return syms


def test_exports_every_declared_symbol(L):
    syms = _declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2511_03343_gb300 import sssp
    assert _declared_symbols() <= set(sssp._SIGNATURES)


def test_abi_version(L):
    from paper_2511_03343_gb300 import sssp
    assert sssp.lib().pe_abi_version() == 1


@pytest.mark.parametrize("sigma,p,tol", [(2.094, 4, 1e-11), (10.47, 6, 1e-8), (26.18, 8, 1e-7), (52.4, 6, 1e-6)])
def test_host_pade_matches_oracle(L, sigma, p, tol):
    """The library's FP64 Baker route against the oracle's: same rational function."""
    from paper_2511_03343_gb300 import sssp
    b, a, d0, d = sssp.pade_coefficients(sigma, p)
    plan = O.pade_plan(sigma, p)
    # the same poles (as sets) and the conjugate pairing a_j = conj(b_j)
    for bj in b:
        assert np.min(np.abs(plan.b - bj)) < tol * max(1, abs(bj))
    assert np.allclose(a, np.conj(b))
    lam = np.linspace(-3, 0.5, 101)
    lib_sum = np.full(lam.shape, d0, dtype=complex)
    lib_prod = np.ones(lam.shape, dtype=complex)
    for bj, aj, dj in zip(b, a, d):
        lib_sum += dj / (1 + bj * lam)
        lib_prod *= (1 + aj * lam) / (1 + bj * lam)
    ref = plan.rational(lam)
    assert np.max(np.abs(lib_sum - ref)) < tol * 10
    assert np.max(np.abs(lib_prod - ref)) < tol * 10


def test_host_pade_rejects_bad_order(L):
    from paper_2511_03343_gb300 import sssp
    with pytest.raises(sssp.PEError) as e:
        sssp.pade_coefficients(2.0, 9)
    assert e.value.status == sssp.PE_ERR_ARG


@pytest.mark.parametrize("args", [
    dict(N=100, H=100.0, k0=0.4, dr=5.0, pade_order=4),      # N + 1 not a power of two
    dict(N=3, H=100.0, k0=0.4, dr=5.0, pade_order=4),        # too small
    dict(N=131071, H=100.0, k0=0.4, dr=5.0, pade_order=4),   # too large for this build
    dict(N=255, H=-1.0, k0=0.4, dr=5.0, pade_order=4),
    dict(N=255, H=100.0, k0=0.0, dr=5.0, pade_order=4),
    dict(N=255, H=100.0, k0=0.4, dr=0.0, pade_order=4),
    dict(N=255, H=100.0, k0=0.4, dr=5.0, pade_order=0),
    dict(N=255, H=100.0, k0=0.4, dr=5.0, pade_order=9),
    dict(N=255, H=100.0, k0=0.4, dr=5.0, pade_order=4, neumann_terms=-1),
    dict(N=255, H=100.0, k0=0.4, dr=5.0, pade_order=4, neumann_terms=65),
])
def test_plan_create_validates_before_device_work(L, args):
    """Invalid sizes and values are rejected on the host with PE_ERR_ARG (no CUDA call)."""
    from paper_2511_03343_gb300 import sssp
    with pytest.raises(sssp.PEError) as e:
        sssp.Plan(**args)
    assert e.value.status == sssp.PE_ERR_ARG
    assert sssp.lib().pe_create_error().decode()


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (it is test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2511_03343_gb300")
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|sssp_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_oracle_has_no_product_import():
    txt = open(os.path.join(ROOT, "oracle", "sssp_oracle.py")).read()
    assert "paper_2511_03343_gb300" not in txt


def test_plan_bytes_estimate_grows(L):
    from paper_2511_03343_gb300 import sssp
    a = sssp.plan_bytes_estimate(1023, 6, 1, 0)
    assert sssp.plan_bytes_estimate(4095, 6, 1, 0) > a
    assert sssp.plan_bytes_estimate(1023, 8, 1, 0) > a
    assert sssp.plan_bytes_estimate(1023, 6, 10, 0) > a
    assert sssp.plan_bytes_estimate(1023, 6, 1, 100) - a == 100 * 1023 * 4
    # grids beyond one CTA's shared memory carry the 7 L complex workspace
    big = sssp.plan_bytes_estimate(8191, 6, 1, 0)
    assert big - sssp.plan_bytes_estimate(4095, 6, 1, 0) > 7 * 8192 * 8


def test_server_submit_host_checks(L):
    """Request validation and the budget check happen on the host at submit (no GPU work)."""
    from paper_2511_03343_gb300 import inputs, sssp
    srv = sssp.Server(hbm_budget_bytes=10_000_000, max_live=4, chunk_steps=10)
    s = inputs.munk(N=255, steps=5)
    rid = srv.submit(s, tl_every=1)
    assert srv.state(rid) == 0                     # queued until a step admits it
    big = inputs.munk(N=65535, steps=5)
    with pytest.raises(sssp.PEError) as e:         # can never fit in a 10 MB budget
        srv.submit(big)
    assert e.value.status == sssp.PE_ERR_OOM
    bad = inputs.munk(N=255, steps=5)
    bad.profiles = []
    with pytest.raises(sssp.PEError):
        srv.submit(bad)
    # cancelling a queued request needs no GPU: it leaves the queue and reads as failed
    rid2 = srv.submit(s, tl_every=1)
    srv.cancel(rid2)
    assert srv.state(rid2) == 3
    with pytest.raises(sssp.PEError, match="cancelled"):
        srv.take(rid2)
    with pytest.raises(sssp.PEError):
        srv.cancel(987654)                         # unknown id
    srv.close()


def test_serving_queue_depth_summary():
    """Queue depth over time (host logic of the serving replay): maxima, time-weighted means
    and the decimated trace."""
    from paper_2511_03343_gb300 import serving
    d = serving._depth_summary([(0.1, 2, 5), (0.3, 4, 1), (0.6, 1, 0)])
    assert d["max_live"] == 4 and d["max_queued"] == 5
    # samples stand for 0.1, 0.2 and 0.3 s
    assert abs(d["mean_live"] - (2 * 0.1 + 4 * 0.2 + 1 * 0.3) / 0.6) < 1e-12
    assert abs(d["mean_queued"] - (5 * 0.1 + 1 * 0.2) / 0.6) < 1e-12
    assert d["trace"] == [[0.1, 2, 5], [0.3, 4, 1], [0.6, 1, 0]]
    many = serving._depth_summary([(0.01 * i, i % 7, i % 3) for i in range(1, 1001)], points=24)
    assert len(many["trace"]) == 24 and many["trace"][-1][0] == 10.0
    assert serving._depth_summary([])["trace"] == []


def test_admission_radius_estimate_matches_dense_eigenvalues(L):
    """The serving admission's host FP64 power iteration (pe_neumann_radius_estimate) against
    the spectral radius of the dense Neumann operator -b_j L_j^{-1} V built from the oracle's
    explicit sine matrix (np.linalg.eigvals), for converging and diverging cases."""
    import math
    from oracle import sssp_oracle as O
    from paper_2511_03343_gb300 import inputs
    checked = []
    for N, f, p, c0 in [(255, 31.6, 7, 1500.0), (255, 31.6, 7, 1525.14), (255, 37.7, 7, 1525.14), (127, 60.0, 4, 1500.0)]:
        z = inputs.depth_grid(N, 5000.0)
        V = inputs.n2_from_c(inputs.munk_c(z), c0) - 1.0
        k0 = 2 * math.pi * f / c0
        g = O.Grid(N=N, H=5000.0, k0=k0, dr=25.0)
        plan = O.pade_plan(g.sigma, p)
        S = O.sine_matrix(N)
        for bj in plan.b:
            M = -bj * ((2.0 / (N + 1)) * S @ np.diag(1.0 / (1.0 + bj * g.lam)) @ S) @ np.diag(V)
            exact = np.max(np.abs(np.linalg.eigvals(M)))
            from paper_2511_03343_gb300 import sssp
            est = sssp.neumann_radius_estimate(V, 5000.0, k0, complex(bj))
            # the decision admission takes agrees, and radii near it are accurate
            assert (est >= 0.98) == (exact >= 0.98), (N, f, p, c0, bj, est, exact)
            if exact >= 0.5:
                assert abs(est - exact) <= 0.03 * exact, (N, f, p, c0, bj, est, exact)
        checked.append(max(np.max(np.abs(np.linalg.eigvals(
            -bj * ((2.0 / (N + 1)) * S @ np.diag(1.0 / (1.0 + bj * g.lam)) @ S) @ np.diag(V)))) for bj in plan.b))
    assert max(checked) > 1.0 and min(checked) < 1.0  # both sides of the decision were exercised


def test_server_pacing_host_checks(L):
    """The serving loop's pacing limit is validated on the host (no GPU work)."""
    from paper_2511_03343_gb300 import sssp
    srv = sssp.Server(hbm_budget_bytes=10_000_000, max_live=4, chunk_steps=10)
    srv.set_pacing(1)
    srv.set_pacing(4096)
    for bad in (0, -3, 4097):
        with pytest.raises(sssp.PEError) as e:
            srv.set_pacing(bad)
        assert e.value.status == sssp.PE_ERR_ARG
    srv.close()
    assert sssp.lib().pe_server_set_pacing(None, 8) == sssp.PE_ERR_ARG


def test_shape_entry_points_reject_null_plans(L):
    """The shape and autotuner entry points check their pointers before any device work."""
    import ctypes
    from paper_2511_03343_gb300 import sssp
    lib = sssp.lib()
    n, u = ctypes.c_int(7), ctypes.c_int(7)
    assert lib.pe_plan_set_cluster_shape(None, 8, 0) == sssp.PE_ERR_ARG
    assert lib.pe_plan_get_cluster_shape(None, ctypes.byref(n), ctypes.byref(u)) == sssp.PE_ERR_ARG
    assert lib.pe_plan_set_shape(None, 8) == sssp.PE_ERR_ARG
    assert lib.pe_march_batch_autotune(None, 1, 4, None, None, None) == sssp.PE_ERR_ARG
    assert sssp.SHAPE_NAMES[3:] == ("cluster8_pull", "cluster8_push", "cluster16_pull", "cluster16_push")
    assert len(sssp.SHAPE_NAMES) == 7  # PE_AUTOTUNE_SHAPES in include/sssp.h
