"""GPU parity of the CUDA marcher against the FP64 oracle, through the C ABI.

Tolerances: the field relative L2 error <= 1e-4 and |TL_gpu - TL_oracle| <= 0.1 dB wherever the
oracle's TL < 100 dB (the stated bar for complex64 fields).  Transform-level checks use the
FP32 rounding bound of a length-L FFT (a few 1e-6 relative).
"""
import math
import os

import numpy as np
import pytest

from oracle import sssp_oracle as O
from paper_2511_03343_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
TL_TOL = 0.1


@pytest.fixture(scope="module")
def sssp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_03343_gb300 import build
    build.build()
    from paper_2511_03343_gb300 import sssp as S
    S.lib()
    return S


def _oracle(s, steps=None, tl_every=1, form="product"):
    """The oracle march.  The GPU marches the product form; the paper's Algorithm 1 writes the
    sum form.  The two are the same operator once the Neumann series has converged (pin P7),
    but a series cut short by the term limit (few terms, or a slowly converging low-frequency
    case) is a different approximation in each form, so by default the GPU is compared with
    the oracle's product form; converged workloads are also compared with the sum form."""
    g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr, bc=getattr(s, "bc", "dirichlet"))
    return O.march(s.u0, s.profiles, g, s.pade_order, steps or s.steps, s.neumann_terms, s.neumann_tol,
                   r0=s.r0, tl_every=tl_every, form=form)


def _gpu(sssp, s, steps=None, tl_every=1, kernel="auto"):
    pl = sssp.plan_for(s, tl_every=tl_every)
    pl.set_kernel(kernel)
    pl.march(steps or s.steps)
    u = pl.read_field()
    tl, rng = pl.read_tl()
    nd = pl.transform_count()
    pl.close()
    return u, tl, rng, nd


def _compare(u, tl, ref, field_tol=FIELD_TOL, tl_tol=TL_TOL):
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= field_tol, f"field rel L2 {rel:.3e}"
    if ref.tl.size:
        assert tl.shape == ref.tl.shape
        mask = ref.tl < 100
        dtl = np.max(np.abs(tl.astype(np.float64) - ref.tl)[mask])
        assert dtl <= tl_tol, f"max TL error {dtl:.3e} dB"
    return rel


# ----------------------------------------------------------------------------- S2/S4 transform
@pytest.mark.parametrize("N", [7, 15, 31, 63, 127, 255, 511, 1023, 2047, 4095])
def test_dst1_matches_oracle(sssp, N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)
    X = pl.dst1(x.astype(np.complex64))
    ref = O.dst1(x)
    err = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
    assert err < 2e-6 * math.log2(N + 1), err
    # DST-I is its own inverse up to 2/(N+1).  The one-CTA transform's odd outputs are prefix
    # sums of L/2 rounded terms (the scan form), so the round trip's FP32 error grows like
    # sqrt(L), not like log2(L) (5.0e-5 measured at N = 4095, where the bound is 6.4e-5)
    back = pl.dst1(X) * (2.0 / (N + 1))
    assert np.max(np.abs(back - x)) / np.max(np.abs(x)) < 1e-6 * max(math.sqrt(N + 1), 4 * math.log2(N + 1))
    pl.close()


@pytest.mark.parametrize("N", [8191, 16383, 32767, 65535])
def test_dst1_large_sampled(sssp, N):
    """Grids beyond one CTA's shared memory: sampled outputs against the oracle's explicit sums."""
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)
    X = pl.dst1(x.astype(np.complex64))
    pl.close()
    ms = np.concatenate([[1, 2, 3, N // 2, N // 2 + 1, N - 1, N], rng.integers(1, N + 1, 25)])
    ref = O.dst1_at(x, ms)
    scale = np.sqrt(N / 2.0) * np.sqrt(2.0)  # typical |X_m| for unit-variance complex input
    err = np.max(np.abs(X[ms - 1] - ref)) / scale
    assert err < 2e-6 * math.log2(N + 1), err


def test_dst1_single_mode(sssp):
    """A sampled sine mode transforms to ((N+1)/2) delta (the closed form)."""
    N, m0 = 1023, 37
    n = np.arange(1, N + 1)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)
    X = pl.dst1(np.sin(np.pi * n * m0 / (N + 1)).astype(np.complex64))
    ref = np.zeros(N)
    ref[m0 - 1] = (N + 1) / 2
    assert np.max(np.abs(X - ref)) < 1e-3
    pl.close()


# ----------------------------------------------------------------------------- workloads
def test_isovelocity_full(sssp):
    """Isovelocity Dirichlet guide, N = 255, 1000 steps of 5 m, [4/4], no Neumann terms."""
    s = inputs.isovelocity()
    u, tl, _, nd = _gpu(sssp, s)
    ref = _oracle(s, form="sum")
    _compare(u, tl, ref)
    assert nd == s.steps + 1  # one TL transform per step + the final field


def test_munk_short(sssp):
    """Range-independent Munk, N = 1023, f = 50 Hz, [6/6], Neumann 1e-10 / 12 terms, 150 steps."""
    s = inputs.munk(N=1023, steps=150)
    u, tl, _, _ = _gpu(sssp, s)
    _compare(u, tl, _oracle(s, form="sum"))   # converged series: Algorithm 1's sum form
    _compare(u, tl, _oracle(s))


@pytest.mark.parametrize("kernel", ["auto", "cta"])
def test_munk_full_size_against_stored_oracle(sssp, kernel):
    """The full Munk workload (N = 4095, 2000 steps) against the stored FP64 oracle runs: the
    product form the GPU marches (tests/golden/munk_n4095_s2000_product.txt; field and TL bars)
    and Algorithm 1's sum form (munk_n4095_s2000.txt; TL bar).  The 12-term series does not
    reach 1e-10 here, so the two forms differ by ~8.5e-5 in the field after 2000 steps."""
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    runs = {form: mg.load(os.path.join(here, name))
            for form, name in (("product", "munk_n4095_s2000_product.txt"), ("sum", "munk_n4095_s2000.txt"))}
    s = inputs.munk()
    pl = sssp.plan_for(s, tl_every=int(runs["product"][0]["tl_every"]))
    pl.set_kernel(kernel)
    pl.march(s.steps)
    u = pl.read_field()
    tl, rng = pl.read_tl()
    pl.close()
    err = {}
    for form, (meta, fidx, fref, tl_r, tl_ref) in runs.items():
        assert np.allclose(rng, tl_r)
        rel = np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)
        tsub = tl[:, ::int(meta["tl_stride"])].astype(np.float64)
        mask = tl_ref < 100
        err[form] = (rel, np.max(np.abs(tsub - tl_ref)[mask]))
        print(f"munk N=4095 2000 steps ({kernel}) vs the {form} form: sampled field rel-L2 {rel:.3e}, "
              f"max TL error {err[form][1]:.4f} dB")
    assert abs(np.linalg.norm(u) / runs["product"][0]["norm"] - 1) < 1e-4
    assert err["product"][0] <= FIELD_TOL and err["product"][1] <= TL_TOL
    assert err["sum"][0] <= FIELD_TOL and err["sum"][1] <= TL_TOL


@pytest.mark.parametrize("kernel", ["auto", "cta", "cluster8"])
def test_eddy_full_length_against_stored_oracle(sssp, kernel):
    """The range-dependent workload at full length (N = 16383, 4000 steps of 25 m, [8/8], a
    profile node per step) against the stored FP64 oracle runs (library DST-I backend):
    tests/golden/eddy_n16383_s4000.txt in the product form the GPU marches (field and TL bars),
    and eddy_n16383_s4000_sum.txt in Algorithm 1's sum form (TL bar).  The 12-term Neumann
    series does not reach 1e-10 on this workload, so the two forms differ (about 1e-3 in the
    field after 4000 steps, in FP64); the TL bar holds against both."""
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    s = inputs.munk_eddy()
    runs = {form: mg.load(os.path.join(here, name))
            for form, name in (("product", "eddy_n16383_s4000.txt"), ("sum", "eddy_n16383_s4000_sum.txt"))}
    meta = runs["product"][0]
    pl = sssp.plan_for(s, tl_every=int(meta["tl_every"]))
    if kernel == "cluster8":  # 8-CTA clusters pushing the exchange (auto: 16 CTAs pulling)
        pl.set_kernel("cluster")
        pl.set_cluster_shape(8, 1)
    else:
        pl.set_kernel(kernel)
    pl.march(s.steps)
    u = pl.read_field()
    tl, rng = pl.read_tl()
    pl.close()
    err = {}
    for form, (meta, fidx, fref, tl_r, tl_ref) in runs.items():
        assert np.allclose(rng, tl_r)
        rel = np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)
        tsub = tl[:, ::int(meta["tl_stride"])].astype(np.float64)
        mask = tl_ref < 100
        err[form] = (rel, np.max(np.abs(tsub - tl_ref)[mask]))
        print(f"eddy N=16383 4000 steps ({kernel}) vs the {form} form: sampled field rel-L2 {rel:.3e}, "
              f"max TL error {err[form][1]:.4f} dB")
    assert abs(np.linalg.norm(u) / runs["product"][0]["norm"] - 1) < 1e-4
    assert err["product"][0] <= FIELD_TOL
    assert err["product"][1] <= TL_TOL
    assert err["sum"][1] <= TL_TOL and err["sum"][0] <= 2e-3


def test_munk_n65535_against_stored_oracle(sssp):
    """The largest grid at range: Munk N = 65535, 500 Hz, [6/6], 12 terms, 2000 steps of 25 m on
    its default kernel (one CTA, two-pass tiled DST) against the stored FP64 oracle run in the
    product form (tests/golden/munk_n65535_s2000.txt): sampled final field and TL rows."""
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    meta, fidx, fref, tl_r, tl_ref = mg.load(os.path.join(here, "munk_n65535_s2000.txt"))
    s = inputs.munk(N=65535, freq=500.0, dr=25.0, steps=2000)
    pl = sssp.plan_for(s, tl_every=int(meta["tl_every"]))
    assert pl.kernel == "cta"
    pl.march(s.steps)
    u = pl.read_field()
    tl, rng = pl.read_tl()
    pl.close()
    assert np.allclose(rng, tl_r)
    rel = np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)
    tsub = tl[:, ::int(meta["tl_stride"])].astype(np.float64)
    mask = tl_ref < 100
    dtl = np.max(np.abs(tsub - tl_ref)[mask])
    print(f"munk N=65535 2000 steps: sampled field rel-L2 {rel:.3e}, max TL error {dtl:.4f} dB")
    assert abs(np.linalg.norm(u) / meta["norm"] - 1) < 1e-4
    assert rel <= FIELD_TOL, rel
    assert dtl <= TL_TOL


def test_range_dependent_eddy(sssp):
    """Munk + Gaussian eddy with a profile node per step (midpoint rule), N = 511, 100 Hz, [8/8].
    The eddy is centred inside the marched range so the profile changes every step."""
    s = inputs.munk_eddy(N=511, freq=100.0, dr=25.0, steps=80, seed=3)
    z = s.z
    cm = inputs.munk_c(z)
    s.profiles = [(n * s.dr, inputs.n2_from_c(cm + inputs.gaussian_eddy_dc((n + 0.5) * s.dr, z, s.eddy_dc, r0=1000.0,
                                                                            Lr=600.0), s.c0))
                  for n in range(s.steps)]
    u, tl, _, _ = _gpu(sssp, s)
    ref = _oracle(s)
    # the oracle run itself is inside the Neumann series' convergence region
    assert abs(np.linalg.norm(ref.u) / np.linalg.norm(s.u0) - 1) < 1e-7
    _compare(u, tl, ref)


@pytest.mark.parametrize("kernel", ["auto", "cta"])
def test_munk_large_grid_short(sssp, kernel):
    """Munk on N = 8191, 100 Hz, [6/6], 12 terms, 8 steps, on the cluster kernel (auto) and on
    the one-CTA global-workspace kernel."""
    s = inputs.munk(N=8191, freq=100.0, dr=25.0, steps=8)
    u, tl, _, _ = _gpu(sssp, s, kernel=kernel)
    ref = _oracle(s)
    _compare(u, tl, ref)


@pytest.mark.parametrize("kernel", ["auto", "cta"])
def test_eddy_n16383_short(sssp, kernel):
    """The range-dependent workload's grid and Pade order (N = 16383, 250 Hz, [8/8], dr = 25 m,
    profile node per step) for its first 3 steps against the oracle, on both kernels."""
    s = inputs.munk_eddy(steps=3)
    u, tl, _, _ = _gpu(sssp, s, kernel=kernel)
    ref = _oracle(s)
    _compare(u, tl, ref)


def test_isovelocity_mode_n65535(sssp):
    """N = 65535, isovelocity: a single sine mode is an eigenvector of the step, so after n steps
    it is (e^{i sigma} R(lambda_m))^n times itself (closed form, any size)."""
    N, m0, steps = 65535, 40, 30
    s = inputs.isovelocity(N=N, H=5000.0, freq=200.0, dr=25.0, steps=steps, pade_order=8)
    z = s.z
    s.u0 = np.sin(np.pi * m0 * z / s.H).astype(np.complex128)
    pl = sssp.plan_for(s)
    pl.march(steps)
    u = pl.read_field()
    pl.close()
    plan = O.pade_plan(s.k0 * s.dr, 8)
    lam = -(np.pi * m0 / (s.k0 * s.H)) ** 2
    G = np.exp(1j * s.k0 * s.dr) * plan.rational(lam)
    ref = G ** steps * s.u0
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("N,p,terms", [(7, 1, 12), (15, 8, 12), (31, 4, 3), (63, 6, 12), (127, 2, 12)])
def test_small_grids_and_orders(sssp, N, p, terms):
    """Tiny grids (partial warps, a single thread for N = 7), Pade orders 1..8, few terms."""
    s = inputs.munk(N=N, freq=10.0, dr=50.0, steps=40, pade_order=p, neumann_terms=terms)
    # an O(1) field made of the low sine modes (the 10 Hz Gaussian is below the grid scale)
    n = np.arange(1, N + 1)
    s.u0 = sum(np.sin(np.pi * n * m / (N + 1)) * (1.0 + 0.5j * m) / m for m in range(1, min(N, 5) + 1))
    u, tl, _, _ = _gpu(sssp, s)
    ref = _oracle(s)
    _compare(u, tl, ref)


def test_truncated_series_is_product_form(sssp):
    """Three Neumann terms (M = 2, the paper's Fig. 1c setting) on a Munk guide: the GPU's
    product form matches the oracle's product form, and differs from the sum form by the
    truncation error (so the two oracle forms are distinguishable here)."""
    s = inputs.munk(N=511, freq=200.0, dr=25.0, steps=60, neumann_terms=3)
    u, tl, _, _ = _gpu(sssp, s)
    ref = _oracle(s, form="product")
    _compare(u, tl, ref)
    other = _oracle(s, form="sum", tl_every=0)
    assert np.linalg.norm(other.u - ref.u) / np.linalg.norm(ref.u) > 1e-3


def test_single_term_ignores_profile(sssp):
    """neumann_terms = 1 keeps only t_0: the isovelocity step with V ignored (Fig. 1a)."""
    s = inputs.munk(N=255, freq=25.0, steps=50, neumann_terms=1)
    u, tl, _, _ = _gpu(sssp, s)
    iso = inputs.munk(N=255, freq=25.0, steps=50, neumann_terms=1)
    iso.profiles = [(0.0, np.ones(255))]
    ref = _oracle(iso)
    _compare(u, tl, ref)


# ----------------------------------------------------------------------------- API behaviour
def test_marches_compose_bitwise(sssp):
    s = inputs.munk(N=511, freq=30.0, steps=30)
    a = sssp.plan_for(s, tl_every=1)
    a.march(30)
    ua = a.read_field()
    tla, ra = a.read_tl()
    b = sssp.plan_for(s, tl_every=1)
    b.march(10)
    b.march(20)
    ub = b.read_field()
    tlb, rb = b.read_tl()
    assert np.array_equal(ua, ub) and np.array_equal(tla, tlb) and np.array_equal(ra, rb)
    assert b.range() == (30 * s.dr, 30)


def test_tl_decimation(sssp):
    s = inputs.isovelocity(steps=50)
    pl = sssp.plan_for(s, tl_every=7)
    pl.march(50)
    tl, rng = pl.read_tl()
    ref = _oracle(s, tl_every=7)
    assert tl.shape == (7, s.N)
    assert np.allclose(rng, ref.tl_ranges)
    assert np.max(np.abs(tl - ref.tl)[ref.tl < 100]) <= TL_TOL


def test_batch_alone_vs_mix(sssp):
    """Uneven sizes and frequencies in one batched march give the same bits as alone."""
    solves = [inputs.munk(N=255, freq=20.0, steps=25), inputs.munk(N=1023, freq=45.0, steps=25),
              inputs.munk(N=255, freq=33.0, steps=25, pade_order=4), inputs.isovelocity(N=511, steps=25)]
    alone = []
    for s in solves:
        pl = sssp.plan_for(s, tl_every=5)
        pl.march(25)
        alone.append((pl.read_field(), pl.read_tl()[0]))
        pl.close()
    plans = [sssp.plan_for(s, tl_every=5) for s in solves]
    sssp.march_batch(plans, 25)
    for pl, (u, tl) in zip(plans, alone):
        assert np.array_equal(pl.read_field(), u)
        assert np.array_equal(pl.read_tl()[0], tl)
        pl.close()


def test_state_errors(sssp):
    pl = sssp.Plan(255, 5000.0, 0.2, 50.0, 6, 12)
    with pytest.raises(sssp.PEError) as e:
        pl.march(1)
    assert e.value.status == sssp.PE_ERR_STATE
    pl.set_field(np.ones(255, dtype=np.complex64))
    with pytest.raises(sssp.PEError) as e:
        pl.march(1)  # Neumann terms requested but no profile
    assert e.value.status == sssp.PE_ERR_STATE
    pl.set_profile(np.ones(255), 100.0)
    with pytest.raises(sssp.PEError) as e:
        pl.set_profile(np.ones(255), 50.0)  # decreasing range
    assert e.value.status == sssp.PE_ERR_ARG
    with pytest.raises(sssp.PEError) as e:
        pl._c(sssp.lib().pe_set_profile(pl.handle, np.full(255, np.nan).ctypes.data, 0, 200.0, 0))
    assert e.value.status == sssp.PE_ERR_ARG
    pl.close()


def test_neumann_divergence_is_reported(sssp):
    """A profile far outside the Neumann series' convergence region (rho >> 1) makes the term
    norms grow; the kernel stops the march and the host reads PE_ERR_NEUMANN_DIVERGED."""
    N = 63
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, 12, 1e-10)
    pl.set_profile(np.full(N, 40.0), 0.0)
    pl.set_field(np.ones(N, dtype=np.complex64))
    pl.march(3)
    with pytest.raises(sssp.PEError) as e:
        pl.sync()
    assert e.value.status == sssp.PE_ERR_NEUMANN_DIVERGED
    pl.close()


def test_norm_conserved_full_munk(sssp):
    """P5 at full size: for real n^2 the Pade operator is unitary, so ||u|| is conserved over
    the whole 2000-step Munk march (a property that needs no oracle run)."""
    s = inputs.munk()
    pl = sssp.plan_for(s)
    pl.march(s.steps)
    u = pl.read_field()
    pl.close()
    assert abs(np.linalg.norm(u) / np.linalg.norm(s.u0) - 1) < 5e-5


def test_batch_workload_sampled_solves(sssp):
    """The 256-solve Munk batch (N = 1023, f ~ U[50, 500] Hz, dr = 25 m, [6/6], 12 terms) marched in
    one batched launch for 60 steps; three sampled solves (lowest, median and highest frequency)
    against the oracle."""
    solves = inputs.munk_batch(steps=60)
    plans = [sssp.plan_for(s, tl_every=20) for s in solves]
    sssp.march_batch(plans, 60)
    freqs = np.array([s.freq for s in solves])
    for idx in [int(np.argmin(freqs)), int(np.argsort(freqs)[128]), int(np.argmax(freqs))]:
        s = solves[idx]
        u = plans[idx].read_field()
        tl, _ = plans[idx].read_tl()
        ref = _oracle(s, tl_every=20)
        _compare(u, tl, ref)
    for pl in plans:
        pl.close()


def _make_golden():
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def test_batch_full_length_against_stored_oracle(sssp):
    """The whole 256-solve batch (N = 1023, f ~ U[50, 500] Hz, 2000 steps of 25 m, [6/6], 12 terms)
    in one batched march, in the launch configuration the bench times; eight members stored from
    the FP64 oracle's product form (tests/golden/batch_n1023_s2000.txt: the lowest and second
    lowest frequency, then evenly up to the highest; the lowest, 53.7 Hz, is the member whose
    12-term series does not converge) compared element by element on the sampled field and TL
    rows."""
    mg = _make_golden()
    runs = mg.load_batch()
    solves = inputs.munk_batch()
    plans = [sssp.plan_for(s, tl_every=mg.BATCH_TL_EVERY) for s in solves]
    sssp.march_batch(plans, solves[0].steps)
    worst = (0.0, 0.0)
    for i, (freq, fidx, fref, tl_r, tl_ref) in runs.items():
        assert abs(solves[i].freq - freq) < 1e-9
        u = plans[i].read_field()
        tl, rng = plans[i].read_tl()
        assert np.allclose(rng, tl_r)
        rel = np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)
        tsub = tl[:, ::mg.BATCH_TL_STRIDE].astype(np.float64)
        mask = tl_ref < 100
        dtl = float(np.max(np.abs(tsub - tl_ref)[mask]))
        print(f"batch member {i} ({freq:.1f} Hz): sampled field rel-L2 {rel:.3e}, max TL error {dtl:.4f} dB")
        assert rel <= FIELD_TOL and dtl <= TL_TOL, (i, freq, rel, dtl)
        worst = (max(worst[0], rel), max(worst[1], dtl))
    for pl in plans:
        pl.close()


def test_transform_count_matches_oracle_term_counts(sssp):
    """The stop test taken on the GPU (FP64 comparison of FP32 sums of squares) sums the same
    number of Neumann terms as the FP64 oracle: over the first 100 steps of the N = 4095 Munk
    march, the GPU's DST-I count equals the count the oracle's per-step, per-Pade-term term
    counts imply (tests/golden/munk_n4095_counts100.txt): a stage with c >= 2 terms takes one
    transform of t_0, c - 1 forward and c - 2 inverse transforms; plus the final field."""
    mg = _make_golden()
    counts = mg.load_counts()
    per_stage = np.where(counts >= 2, 2 * counts - 2, 1)
    expected = int(per_stage.sum()) + 1
    s = inputs.munk(steps=counts.shape[0])
    for kernel in ("cta", "cluster"):
        pl = sssp.plan_for(s, tl_every=0)
        pl.set_kernel(kernel)
        pl.march(s.steps)
        pl.sync()
        got = pl.transform_count()  # counted by the march kernel (the starter's transform is not)
        pl.close()
        print(f"{kernel}: {got} transforms, oracle term counts imply {expected}")
        assert got == expected, (kernel, got, expected)


# ----------------------------------------------------------------------------- serving loop
def _mixed_trace(seed=7, count=14):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        env = ["isovelocity", "munk", "munk_eddy"][i % 3]
        N = [255, 1023, 4095, 8191][int(rng.integers(0, 4))]
        H = 100.0 if env == "isovelocity" else 5000.0
        out.append(dict(id=i, t_arrival=0.002 * i, N=N, env=env, H=H, freq=float(rng.uniform(25, 60 if H > 1000 else 300)),
                        range_m=float(rng.uniform(300, 1500)), dr=25.0, pade_order=int(rng.integers(4, 9)),
                        zs=0.4 * H, eddy_dc=-20.0, eddy_r0=500.0))
    return out


def test_server_alone_vs_mix_bitwise(sssp):
    """Continuous batching: requests arriving while others run are admitted and share launches;
    every result is bit-identical to marching that request alone."""
    from paper_2511_03343_gb300 import serving
    trace = _mixed_trace()
    res = serving.replay(trace, hbm_budget=64e6, chunk_steps=7, tl_every=5, keep_results=True, admit=0)
    assert len(res["results"]) == len(trace)
    assert res["peak_live"] > 1
    for i, (field, tl, s, _) in res["results"].items():
        pl = sssp.plan_for(s, tl_every=5)
        pl.march(s.steps)
        assert np.array_equal(pl.read_field(), field), i
        assert np.array_equal(pl.read_tl()[0], tl), i
        pl.close()


def test_server_budget_and_parity(sssp):
    """A budget that fits only a few plans at a time: the peak stays within it, everything
    completes, and a served result matches the oracle."""
    from paper_2511_03343_gb300 import serving
    trace = _mixed_trace(seed=8, count=9)
    one = max(sssp.plan_bytes_estimate(t["N"], t["pade_order"], 1, 100) for t in trace)
    budget = 3 * one
    res = serving.replay(trace, hbm_budget=budget, chunk_steps=11, tl_every=0, keep_results=True)
    assert res["peak_bytes"] <= budget
    assert len(res["results"]) == len(trace)
    i = next(i for i, t in enumerate(trace) if t["env"] == "munk" and t["N"] <= 1023)
    field, _, s, prm = res["results"][i]
    ref = _oracle_admitted(s, prm, tl_every=0)
    assert np.linalg.norm(field - ref.u) / np.linalg.norm(ref.u) <= FIELD_TOL


def _oracle_admitted(s, prm, tl_every=1):
    """The oracle march of a served request with the values admission chose: k0, the n^2
    scale (the minimax reference sound speed) and the Pade order."""
    k0, sc, p = prm
    g = O.Grid(N=s.N, H=s.H, k0=k0, dr=s.dr)
    prof = [(r, sc * np.asarray(n2)) for r, n2 in s.profiles]
    return O.march(s.u0, prof, g, p, s.steps, s.neumann_terms, s.neumann_tol, r0=s.r0, tl_every=tl_every,
                   form="product")


def test_server_admission_makes_diverging_requests_converge(sssp):
    """Requests of the serving trace (low frequency, coarse grid, Pade order 7-8) whose 12-term
    Neumann series contracts too slowly: with c0 = 1500 m/s and the minimax c0 alone their march
    grows until it is no longer finite; admission then lowers the Pade order until the cut
    series is accurate, and every request completes and matches the oracle marched with the
    same values (field <= 1e-4, TL <= 0.1 dB)."""
    from paper_2511_03343_gb300 import serving
    trace = inputs.serving_trace(count=1000)
    ids = [2, 15, 768]
    sub = []
    for k, i in enumerate(ids):
        t = dict(trace[i])
        t["t_arrival"] = 0.001 * k
        t["range_m"] = 20000.0
        sub.append(t)
    only_c0 = serving.replay(sub, hbm_budget=4e9, chunk_steps=50, tl_every=10, admit=sssp.ADMIT_MINIMAX_C0)
    print("minimax c0 alone:", only_c0["failed"], "of", len(sub), "failed", only_c0["failures"])
    res = serving.replay(sub, hbm_budget=4e9, chunk_steps=50, tl_every=10, keep_results=True)
    assert res["failed"] == 0, res["failures"]
    assert res["order_lowered"] == len(sub)
    for i, (field, tl, s, prm) in res["results"].items():
        assert np.all(np.isfinite(field))
        assert prm[2] < s.pade_order
        ref = _oracle_admitted(s, prm, tl_every=10)
        _compare(field, tl, ref)


# ----------------------------------------------------------------------------- tensor-core GEMM-DST
def test_gemm_dst_small_against_fft_marcher(sssp):
    """The tensor-core GEMM-DST batch (own tcgen05 kernels) on a small case first: 20 Munk solves
    at N = 255 (two 128-row tiles, two 32-column tiles), [2/2], a fixed 3 terms (tolerance 0 in
    both marchers), 3 steps, against the FFT marcher with the same fixed term count."""
    freqs = np.linspace(40.0, 120.0, 20)
    solves = [inputs.munk(N=255, freq=float(f), dr=25.0, steps=3, pade_order=2, neumann_terms=3, neumann_tol=0.0)
              for f in freqs]
    refs = []
    for s in solves:
        pl = sssp.plan_for(s)
        pl.march(3)
        refs.append(pl.read_field())
        pl.close()
    bars = {"fp32": 1e-5, "3xtf32": 1e-5, "bf16x3": 1e-4, "tf32": 5e-3}
    for mode, bar in bars.items():
        plans = [sssp.plan_for(s) for s in solves]
        gb = sssp.GemmBatch(plans, mode)
        gb.march(3)
        e = max(np.linalg.norm(gb.read_field(i) - r) / np.linalg.norm(r) for i, r in enumerate(refs))
        gb.close()
        for pl in plans:
            pl.close()
        print(f"GEMM-DST {mode}: max field rel-L2 vs the FFT marcher after 3 steps {e:.3e}")
        assert e <= bar, (mode, e)


def test_gemm_dst_precisions(sssp):
    """The batched march with the DST-I as a dense GEMM, per precision, against the FP64 oracle
    (6 Munk solves, N = 1023, 60-200 Hz, dr = 25 m, [6/6], 12 terms, 40 steps).  FP32, the
    3xTF32 split and the BF16x3 split meet the field tolerance; plain TF32 (10-bit mantissa)
    cannot.  The errors are printed for the record."""
    freqs = [60.0, 80.0, 100.0, 130.0, 160.0, 200.0]
    solves = [inputs.munk(N=1023, freq=f, dr=25.0, steps=40) for f in freqs]
    refs = [_oracle(s, tl_every=0).u for s in solves]
    errs = {}
    for mode in ["fp32", "3xtf32", "bf16x3", "tf32"]:
        plans = [sssp.plan_for(s) for s in solves]
        gb = sssp.GemmBatch(plans, mode)
        gb.march(40)
        e = []
        for i, ref in enumerate(refs):
            u = gb.read_field(i)
            e.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
        gb.close()
        for pl in plans:
            pl.close()
        errs[mode] = max(e)
    print("GEMM-DST max field rel-L2 after 40 steps:", errs)
    assert errs["fp32"] <= FIELD_TOL and errs["3xtf32"] <= FIELD_TOL and errs["bf16x3"] <= FIELD_TOL
    assert errs["tf32"] > errs["3xtf32"]


# Full-length error of the tensor-core splits (measured on the GB300, worst of the 8 stored members,
# K split in two halves summed in FP32): BF16x3 3.5e-3 field / 0.054 dB TL, 3xTF32 7.1e-3 / 0.11 dB
# (7.4e-3 / 0.14 and 1.4e-2 / 0.26 with one accumulator over the whole of K).  They do not reach
# the 1e-4 bar over 2000 steps: each transform carries a systematic error (the BF16
# representation of S, 2e-6 relative, and the tensor-core accumulation, ~2.6e-6 per transform
# where exact accumulation of the same 3xTF32 operands gives 7e-8) that adds up coherently over
# ~2.6e5 transforms.  The bounds below (twice the measured figures) guard them against regressions.
GEMM_FULL_BOUNDS = {"bf16x3": (7e-3, 0.11), "3xtf32": (1.5e-2, 0.23)}


@pytest.mark.parametrize("mode", ["bf16x3", "3xtf32"])
def test_gemm_dst_full_batch_against_stored_oracle(sssp, mode):
    """The whole 256-solve batch (N = 1023, 2000 steps of 25 m, [6/6], 12 terms) with the DST-I
    as the tensor-core GEMM in a split precision, against the stored FP64 oracle runs of eight
    members with the same rule, a fixed 12 terms per step (tests/golden/batch_n1023_s2000_fixed12.txt;
    in FP64 it differs from the 1e-10 stop rule by ~1e-9): sampled final field and its TL
    against the stored last TL row, within the measured bounds of GEMM_FULL_BOUNDS."""
    mg = _make_golden()
    runs = mg.load_batch(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "batch_n1023_s2000_fixed12.txt"))
    solves = inputs.munk_batch()
    plans = [sssp.plan_for(s) for s in solves]
    gb = sssp.GemmBatch(plans, mode)
    gb.march(solves[0].steps)
    worst = (0.0, 0.0)
    for i, (freq, fidx, fref, tl_r, tl_ref) in runs.items():
        u = gb.read_field(i).astype(np.complex128)
        rel = np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)
        tl = O.transmission_loss(u, tl_r[-1])[::mg.BATCH_TL_STRIDE]
        mask = tl_ref[-1] < 100
        dtl = float(np.max(np.abs(tl - tl_ref[-1])[mask]))
        print(f"GEMM-DST {mode} member {i} ({freq:.1f} Hz): field rel-L2 {rel:.3e}, final TL error {dtl:.4f} dB")
        worst = (max(worst[0], rel), max(worst[1], dtl))
    gb.close()
    for pl in plans:
        pl.close()
    fb, tb = GEMM_FULL_BOUNDS[mode]
    assert worst[0] <= fb and worst[1] <= tb, worst


@pytest.mark.parametrize("N,count", [(255, 7), (4095, 3), (16383, 2)])
def test_dst1_batch_equals_single(sssp, N, count):
    """The batched DST entry gives every field the same bits as the single-field one."""
    import torch
    rng = np.random.default_rng(N + count)
    x = (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))).astype(np.complex64)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)
    d_in = torch.from_numpy(x).cuda()
    d_out = torch.empty_like(d_in)
    pl.dst1_batch(d_in, d_out)
    got = d_out.cpu().numpy()
    for b in range(count):
        assert np.array_equal(got[b], pl.dst1(x[b]))
    pl.close()


@pytest.mark.parametrize("N", [511, 8191, 16383])
def test_absorbing_layer(sssp, N):
    """Complex n^2 (Section 3.1's complex absorbing potential) in the bottom 20 % of a Munk guide:
    the march matches the oracle and the field's norm decreases (energy leaves through the layer).
    N = 8191 runs the 8-CTA cluster kernel with a complex profile, N = 16383 the 16-CTA one."""
    s = inputs.munk(N=N, freq=60.0 if N < 4096 else 100.0, dr=25.0, steps=40 if N < 4096 else (6 if N < 16383 else 3))
    z = s.z
    za = 0.8 * s.H
    n2 = s.profiles[0][1].astype(np.complex128) + 1j * 0.02 * np.clip((z - za) / (s.H - za), 0.0, None) ** 2
    s.profiles = [(0.0, n2)]
    s.u0 = s.u0 + inputs.gaussian_starter(z, s.k0, 0.9 * s.H)  # energy that reaches the layer
    u, tl, _, _ = _gpu(sssp, s)
    ref = _oracle(s)
    _compare(u, tl, ref)
    assert np.linalg.norm(u) < 0.999 * np.linalg.norm(s.u0)


# ----------------------------------------------------------------------------- periodic boundaries
@pytest.mark.parametrize("N", [8, 64, 256, 4096])
def test_dft_periodic_plan(sssp, N):
    """A periodic plan's transform is the DFT (Section 3's Fourier inversion)."""
    rng = np.random.default_rng(N + 5)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, bc="periodic")
    X = pl.dst1(x.astype(np.complex64))
    ref = O.dft(x)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 2e-6 * math.log2(N)
    pl.close()


def test_periodic_isovelocity_and_mode(sssp):
    """Periodic isovelocity march (N = 256, 1000 steps) vs the oracle, and a single Fourier mode
    e^{2 pi i 7 z/H} at N = 4096 against its closed form."""
    s = inputs.isovelocity(N=256, bc="periodic")
    u, tl, _, _ = _gpu(sssp, s)
    _compare(u, tl, _oracle(s))
    s = inputs.isovelocity(N=4096, H=1000.0, freq=150.0, dr=10.0, steps=200, pade_order=6, bc="periodic")
    s.u0 = np.exp(2j * np.pi * 7 * s.z / s.H)
    pl = sssp.plan_for(s)
    pl.march(s.steps)
    u = pl.read_field()
    pl.close()
    plan = O.pade_plan(s.k0 * s.dr, 6)
    G = np.exp(1j * s.k0 * s.dr) * plan.rational(-(2 * np.pi * 7 / (s.k0 * s.H)) ** 2)
    assert np.linalg.norm(u - G ** s.steps * s.u0) / np.linalg.norm(s.u0) < 1e-5


@pytest.mark.parametrize("N", [512, 4096])
def test_periodic_munk(sssp, N):
    """Munk profile on a periodic grid with the Neumann series, vs the oracle's periodic march."""
    s = inputs.munk(N=N, freq=50.0 if N > 1000 else 30.0, dr=50.0, steps=60 if N < 4096 else 20, bc="periodic")
    u, tl, _, _ = _gpu(sssp, s)
    _compare(u, tl, _oracle(s))


# ----------------------------------------------------------------------------- physics beyond parity
def test_modal_starter_against_normal_modes(sssp):
    """Range-independent Munk (N = 1023, 50 Hz, [6/6], dr = 50 m, 100 steps) from the paper's
    normal-mode starter (modes within 30 degrees of horizontal): the GPU march agrees with the
    normal-mode (exact one-way) field, the reference of Section 4.1, within the Pade and FP32
    errors, and with the oracle march."""
    s = inputs.munk(N=1023, freq=50.0, dr=50.0, steps=100)
    z = s.z
    s.u0 = inputs.modal_starter(z, s.H, inputs.munk_c(z), s.freq, s.zs, max_angle_deg=30.0)
    u, tl, _, _ = _gpu(sssp, s)
    ref = _oracle(s)
    _compare(u, tl, ref)
    g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr)
    modes = O.modal_field(s.u0, g, s.profiles[0][1], s.steps * s.dr)
    assert np.linalg.norm(u - modes) / np.linalg.norm(modes) < 2e-5


# ----------------------------------------------------------------------------- Neumann boundaries
@pytest.mark.parametrize("N", [9, 65, 1025, 2049])
def test_dct1_neumann_plan(sssp, N):
    """A Neumann plan's transform is the DCT-I (computed on the GPU as half the DFT of the even
    extension)."""
    rng = np.random.default_rng(N + 9)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, bc="neumann")
    X = pl.dst1(x.astype(np.complex64))
    ref = O.dct1(x)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 2e-6 * math.log2(2 * (N - 1))
    pl.close()


def test_neumann_mode_and_munk(sssp):
    """Neumann boundaries: a single mode cos(pi 5 z/H) against its closed form, and a Munk march
    (N = 1025, [6/6], Neumann series) against the oracle's DCT-I march."""
    s = inputs.isovelocity(N=513, H=1000.0, freq=150.0, dr=10.0, steps=100, pade_order=6, bc="neumann")
    s.u0 = np.cos(np.pi * 5 * s.z / s.H).astype(np.complex128)
    pl = sssp.plan_for(s)
    pl.march(s.steps)
    u = pl.read_field()
    pl.close()
    plan = O.pade_plan(s.k0 * s.dr, 6)
    G = np.exp(1j * s.k0 * s.dr) * plan.rational(-(np.pi * 5 / (s.k0 * s.H)) ** 2)
    assert np.linalg.norm(u - G ** s.steps * s.u0) / np.linalg.norm(s.u0) < 1e-5
    s = inputs.munk(N=1025, freq=60.0, dr=50.0, steps=40, bc="neumann")
    u, tl, _, _ = _gpu(sssp, s)
    _compare(u, tl, _oracle(s))


# ----------------------------------------------------------------------------- checkpoint / resume
@pytest.mark.parametrize("case", ["munk_dirichlet", "periodic", "neumann", "large"])
def test_checkpoint_resume_bitwise(sssp, case):
    """Saving the spectral state after k steps, loading it into a fresh plan and marching the
    rest gives the same bits (field and the TL rows after the resume) as one uninterrupted march."""
    if case == "munk_dirichlet":
        s = inputs.munk(N=1023, freq=100.0, dr=25.0, steps=40)
    elif case == "periodic":
        s = inputs.munk(N=1024, freq=100.0, dr=25.0, steps=40, bc="periodic")
    elif case == "neumann":
        s = inputs.munk(N=1025, freq=100.0, dr=25.0, steps=40, bc="neumann")
    else:
        s = inputs.munk(N=8191, freq=100.0, dr=25.0, steps=6)
    k = s.steps // 2
    ref = sssp.plan_for(s, tl_every=1)
    ref.march(s.steps)
    u_ref = ref.read_field()
    tl_ref, _ = ref.read_tl()
    ref.close()
    a = sssp.plan_for(s, tl_every=1)
    a.march(k)
    u_k = a.read_field()
    state, r_set, steps = a.save_state()
    assert steps == k and state.size == sssp.lib().pe_state_size(a._p) // 2
    a.close()
    b = sssp.plan_for(s, tl_every=1)
    b.load_state(state, r_set, steps)
    assert np.array_equal(b.read_field(), u_k)
    b.march(s.steps - k)
    assert b.range()[1] == s.steps
    assert np.array_equal(b.read_field(), u_ref)
    tl_b, rng_b = b.read_tl()
    assert np.array_equal(tl_b, tl_ref[k:])
    assert np.allclose(rng_b, s.r0 + s.dr * np.arange(k + 1, s.steps + 1))
    b.close()


def test_load_state_argument_checks(sssp):
    s = inputs.munk(N=255, steps=3)
    pl = sssp.plan_for(s)
    with pytest.raises(sssp.PEError):
        pl.load_state(np.zeros(256, np.complex64), 0.0, -1)
    with pytest.raises(sssp.PEError):
        pl.load_state(np.zeros(256, np.complex64), float("nan"), 0)
    pl.close()
    fresh = sssp.Plan(255, 5000.0, 0.2, 25.0, 4)
    with pytest.raises(sssp.PEError):              # nothing to save before a field is set
        fresh.save_state()
    fresh.close()


# ----------------------------------------------------------------------------- Neumann bound, status
@pytest.mark.parametrize("bc,N", [("dirichlet", 1023), ("periodic", 1024), ("neumann", 1025)])
def test_neumann_bound_matches_oracle(sssp, bc, N):
    """The library's host bound on the Neumann series (from the device copy of V) against the
    oracle's, per Pade term; V is FP32 on the device, hence the 1e-6 relative tolerance."""
    s = inputs.munk(N=N, freq=60.0, dr=25.0, steps=2, bc=bc)
    pl = sssp.plan_for(s)
    rho = pl.neumann_bound(0)
    g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr, bc=bc)
    V = O.profile_at(s.profiles, 0.0) - 1.0
    ref = O.neumann_bound(V, O.pade_plan(g.sigma, s.pade_order).b, g.lam)
    assert np.allclose(rho, ref, rtol=1e-6, atol=0), (rho, ref)
    with pytest.raises(sssp.PEError):
        pl.neumann_bound(5)                        # no such node
    pl.close()


def test_injected_device_status_is_reported(sssp):
    """The error path of a failing march, without a failing march: a status word written into
    the plan's device status is reported by the next call that checks it, and a new starter
    clears it."""
    s = inputs.munk(N=255, steps=4)
    pl = sssp.plan_for(s)
    pl.march(2)
    pl.inject_status(4)
    with pytest.raises(sssp.PEError) as e:
        pl.sync()
    assert e.value.status == sssp.PE_ERR_NEUMANN_DIVERGED
    pl.inject_status(7)
    with pytest.raises(sssp.PEError) as e:
        pl.read_field()
    assert e.value.status == sssp.PE_ERR_NUMERIC
    pl.set_field(s.u0, r=s.r0)
    pl.march(4)
    u = pl.read_field()
    pl.close()
    ref = sssp.plan_for(s)
    ref.march(4)
    assert np.array_equal(u, ref.read_field())
    ref.close()


def test_server_cancel_running(sssp):
    """Cancelling a running request frees its budget at once; the others complete unchanged."""
    srv = sssp.Server(hbm_budget_bytes=200_000_000, max_live=8, chunk_steps=5)
    solves = [inputs.munk(N=511, freq=f, dr=25.0, steps=30) for f in (80.0, 100.0, 120.0)]
    ids = [srv.submit(s, tl_every=0) for s in solves]
    srv.step()
    assert all(srv.state(i) == 1 for i in ids)
    before = srv.stats()["bytes_in_use"]
    srv.cancel(ids[1])
    assert srv.state(ids[1]) == 3 and srv.stats()["bytes_in_use"] < before
    while any(srv.state(i) < 2 for i in (ids[0], ids[2])):
        srv.step()
    for i, s in ((ids[0], solves[0]), (ids[2], solves[2])):
        f, _ = srv.take(i)
        pl = sssp.plan_for(s)
        pl.march(s.steps)
        assert np.array_equal(pl.read_field(), f)
        pl.close()
    with pytest.raises(sssp.PEError, match="cancelled"):
        srv.take(ids[1])
    srv.close()


def test_server_pacing_lets_small_grids_finish_first(sssp):
    """Pacing: a cheap request (N = 255) beside a costly one (N = 4095, 24x the work per step)
    marches 24 chunks per server step, so it finishes in the second step instead of the 40th
    (lockstep, pacing 1); both results equal marching alone, bit for bit, either way."""
    small = inputs.munk(N=255, freq=40.0, dr=25.0, steps=400)
    big = inputs.munk(N=4095, freq=50.0, dr=50.0, steps=100)
    ref = []
    for s in (small, big):
        pl = sssp.plan_for(s)
        pl.march(s.steps)
        ref.append(pl.read_field())
        pl.close()

    def run(pacing):
        srv = sssp.Server(hbm_budget_bytes=2_000_000_000, max_live=4, chunk_steps=10)
        srv.set_pacing(pacing)
        a, b = srv.submit(small, tl_every=0), srv.submit(big, tl_every=0)
        n, small_done = 0, None
        while srv.state(a) < 2 or srv.state(b) < 2:
            srv.step()
            n += 1
            if small_done is None and srv.state(a) == 2:
                small_done = n
        fa, _ = srv.take(a)
        fb, _ = srv.take(b)
        srv.close()
        return small_done, n, fa, fb

    paced = run(64)
    lock = run(1)
    assert paced[:2] == (2, 10), paced[:2]
    assert lock[:2] == (40, 40), lock[:2]
    for got in (paced, lock):
        assert np.array_equal(got[2], ref[0]) and np.array_equal(got[3], ref[1])
    srv = sssp.Server(hbm_budget_bytes=1_000_000, max_live=1, chunk_steps=1)
    with pytest.raises(sssp.PEError):
        srv.set_pacing(0)
    srv.close()


# ----------------------------------------------------------------------------- cluster kernel
@pytest.mark.parametrize("N", [4095, 8191, 16383, 32767])
def test_cluster_dst_matches_oracle(sssp, N):
    """The cluster transform (residue rows over 8 or 16 CTAs, local FFTs + one all-to-all, the
    scan-free DST-I) against the oracle: every output at N = 4095, sampled outputs beyond."""
    rng = np.random.default_rng(N + 11)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)
    pl.set_kernel("cluster")
    X = pl.dst1(x.astype(np.complex64))
    pl.close()
    scale = np.sqrt(N / 2.0) * np.sqrt(2.0)
    if N == 4095:
        err = np.max(np.abs(X - O.dst1(x))) / scale
    else:
        ms = np.concatenate([[1, 2, 3, N // 2, N // 2 + 1, N - 1, N], rng.integers(1, N + 1, 40)])
        err = np.max(np.abs(X[ms - 1] - O.dst1_at(x, ms))) / scale
    # the scan-free form has the FFT's error (no prefix scan): a few FP32 ulps times log2 L
    assert err < 1e-6 * math.log2(N + 1), err


def test_cluster_kernel_choice(sssp):
    """Automatic choice: the cluster kernel for Dirichlet N + 1 >= 4096, one CTA below; the
    cluster kernel is refused where it does not apply."""
    big = sssp.Plan(8191, 5000.0, 0.4, 25.0, 6, 12)
    assert big.kernel == "cluster"
    big.set_kernel("cta")
    assert big.kernel == "cta"
    big.close()
    mid = sssp.Plan(4095, 5000.0, 0.4, 25.0, 6, 12)
    assert mid.kernel == "cluster"
    mid.set_kernel("cta")
    assert mid.kernel == "cta"
    mid.close()
    for pl in (sssp.Plan(1023, 5000.0, 0.4, 25.0, 6, 12), sssp.Plan(65535, 5000.0, 0.4, 25.0, 6, 12),
               sssp.Plan(4096, 5000.0, 0.4, 25.0, 6, 12, bc="periodic")):
        with pytest.raises(sssp.PEError) as e:
            pl.set_kernel("cluster")
        assert e.value.status == sssp.PE_ERR_ARG
        pl.close()


def test_cluster_march_n4095_matches_oracle_and_cta(sssp):
    """Munk N = 4095, 100 Hz, [6/6], 12 terms, 30 steps on the cluster kernel: against the
    oracle (field and TL bars) and against the one-CTA kernel (FP32 rounding apart)."""
    s = inputs.munk(N=4095, freq=100.0, dr=25.0, steps=30)
    out = {}
    for k in ("cluster", "cta"):
        pl = sssp.plan_for(s, tl_every=1)
        pl.set_kernel(k)
        pl.march(s.steps)
        out[k] = (pl.read_field(), pl.read_tl()[0], pl.transform_count())
        pl.close()
    ref = _oracle(s)
    rel = _compare(out["cluster"][0], out["cluster"][1], ref)
    print("cluster N=4095 30 steps field rel-L2 vs oracle:", rel)
    d = np.linalg.norm(out["cluster"][0] - out["cta"][0]) / np.linalg.norm(out["cta"][0])
    assert d < 2e-5, d
    # the same Neumann term counts up to stop decisions at the FP32 rounding edge
    assert abs(out["cluster"][2] - out["cta"][2]) <= 0.02 * out["cta"][2]


def test_cluster_isovelocity_mode_n32767(sssp):
    """N = 32767 on the 16-CTA cluster, isovelocity: a sine mode is an eigenvector of the step,
    so after n steps it is (e^{i sigma} R(lambda_m))^n times itself (closed form); the TL rows
    come from the cluster's inverse transform."""
    N, m0, steps = 32767, 57, 25
    s = inputs.isovelocity(N=N, H=5000.0, freq=200.0, dr=25.0, steps=steps, pade_order=8)
    s.u0 = np.sin(np.pi * m0 * s.z / s.H).astype(np.complex128)
    pl = sssp.plan_for(s, tl_every=5)
    assert pl.kernel == "cluster"
    pl.march(steps)
    u = pl.read_field()
    tl, _ = pl.read_tl()
    pl.close()
    plan = O.pade_plan(s.k0 * s.dr, 8)
    G = np.exp(1j * s.k0 * s.dr) * plan.rational(-(np.pi * m0 / (s.k0 * s.H)) ** 2)
    ref = G ** steps * s.u0
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-5
    ref_tl = -20 * np.log10(np.abs(ref)) + 10 * np.log10(s.r0 + s.dr * steps)
    mask = ref_tl < 100
    assert np.max(np.abs(tl[-1][mask] - ref_tl[mask])) < TL_TOL


def test_cluster_munk_n32767_vs_cta(sssp):
    """Munk N = 32767, 300 Hz, [6/6], 12 terms, 4 steps: the 16-CTA cluster kernel against the
    one-CTA global-workspace kernel, and norm conservation for the real profile."""
    s = inputs.munk(N=32767, freq=300.0, dr=25.0, steps=4)
    out = {}
    for k in ("cluster", "cta"):
        pl = sssp.plan_for(s)
        pl.set_kernel(k)
        pl.march(s.steps)
        out[k] = pl.read_field()
        pl.close()
    d = np.linalg.norm(out["cluster"] - out["cta"]) / np.linalg.norm(out["cta"])
    assert d < 1e-5, d
    assert abs(np.linalg.norm(out["cluster"]) / np.linalg.norm(s.u0) - 1) < 1e-5


def test_cluster_divergence_is_reported(sssp):
    """A diverging Neumann series on the cluster kernel: every CTA takes the same stop decision
    (the status is reported, the march ends, the plan stays usable)."""
    N = 4095
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, 12, 1e-10)
    pl.set_kernel("cluster")
    pl.set_profile(np.full(N, 40.0), 0.0)
    pl.set_field(np.ones(N, dtype=np.complex64))
    pl.march(3)
    with pytest.raises(sssp.PEError) as e:
        pl.sync()
    assert e.value.status == sssp.PE_ERR_NEUMANN_DIVERGED
    pl.set_profile(np.full(N, 1.0), 1.0)
    pl.set_field(np.ones(N, dtype=np.complex64))
    pl.march(2)
    pl.sync()
    pl.close()


def test_cluster_batch_alone_vs_mix(sssp):
    """Cluster solves and one-CTA solves in one batched call: each result has the same bits as
    marching it alone."""
    solves = [inputs.munk(N=8191, freq=90.0, dr=25.0, steps=5), inputs.munk(N=1023, freq=60.0, steps=5),
              inputs.munk(N=8191, freq=120.0, dr=25.0, steps=5), inputs.munk(N=16383, freq=200.0, dr=25.0, steps=5)]
    alone = []
    for s in solves:
        pl = sssp.plan_for(s, tl_every=1)
        pl.march(5)
        alone.append((pl.read_field(), pl.read_tl()[0]))
        pl.close()
    plans = [sssp.plan_for(s, tl_every=1) for s in solves]
    assert [p.kernel for p in plans] == ["cluster", "cta", "cluster", "cluster"]
    sssp.march_batch(plans, 5)
    for pl, (u, tl) in zip(plans, alone):
        assert np.array_equal(pl.read_field(), u)
        assert np.array_equal(pl.read_tl()[0], tl)
        pl.close()


# ----------------------------------------------------------------------------- autotuner
def test_autotune_restores_the_march_and_caches(sssp, tmp_path, monkeypatch):
    """pe_plan_autotune in the middle of a march: the march goes on with the same bits as
    marching on the chosen kernel without tuning (state and TL bookkeeping restored), and the
    choice is cached for a plan of the same shape."""
    monkeypatch.setenv("SSSP_TUNE_CACHE", str(tmp_path / "tune.json"))
    s = inputs.munk(N=4095, freq=100.0, dr=25.0, steps=10)
    pl = sssp.plan_for(s, tl_every=1)
    first = pl.kernel
    pl.march(3)
    res = pl.autotune(steps=2)
    assert res["kernel"] in ("cta", "cluster") and not res["cached"]
    assert res["ms_cta"] > 0 and res["ms_cluster"] is not None and res["ms_cluster"] > 0
    assert pl.kernel == res["kernel"]
    pl.march(7)
    u = pl.read_field()
    tl, rng = pl.read_tl()
    pl.close()
    ref = sssp.plan_for(s, tl_every=1)
    ref.set_kernel(first)
    ref.march(3)
    ref.set_kernel(res["kernel"])
    ref.march(7)
    assert np.array_equal(u, ref.read_field())
    tl_ref, rng_ref = ref.read_tl()
    assert np.array_equal(tl, tl_ref) and np.allclose(rng, rng_ref)
    ref.close()
    again = sssp.plan_for(s, tl_every=1)
    res2 = again.autotune(steps=2)
    assert res2["cached"] and res2["kernel"] == res["kernel"] and again.kernel == res["kernel"]
    again.close()
    small = sssp.plan_for(inputs.munk(N=255, steps=4), tl_every=0)  # one candidate only
    r3 = small.autotune(steps=2, cache=False)
    assert r3["kernel"] == "cta" and r3["ms_cluster"] is None
    small.close()


def test_batch_of_two_sizes_overlaps_on_the_device(sssp):
    """A batched march over two grid sizes (N = 255 and N = 65535) runs each size's launch on its
    own stream, forked from and joined to the plan stream: the batch takes less device time than
    the two groups marched one after the other, and each result is the same as marching alone."""
    import torch
    stream = torch.cuda.current_stream()
    small = [inputs.munk(N=255, freq=30.0, dr=25.0, steps=400, pade_order=4) for _ in range(4)]
    large = [inputs.munk(N=65535, freq=300.0, dr=25.0, steps=2, pade_order=4)]
    solves = small + large

    def plans():
        return [sssp.plan_for(s, stream=stream) for s in solves]

    def timed(ps, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sssp.march_batch_steps(ps, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ps = plans()
    timed(ps, [s.steps for s in solves])  # warm-up (tables, attributes)
    ps = plans()
    t_small = timed(ps[:4], [s.steps for s in small])
    t_large = timed(ps[4:], [s.steps for s in large])
    alone = [p.read_field() for p in ps]
    ps2 = plans()
    t_both = timed(ps2, [s.steps for s in solves])
    for a, p in zip(alone, ps2):
        assert np.array_equal(a, p.read_field())
    for p in ps + ps2:
        p.close()
    assert t_both < 0.85 * (t_small + t_large), (t_small, t_large, t_both)



@pytest.mark.parametrize("ppt", [4, 16])
def test_cta_shapes_match_oracle_and_default(sssp, ppt):
    """The one-CTA kernel at 4 and 16 points per thread (pe_plan_set_shape): a short Munk march
    at N = 1023 and N = 4095 against the oracle, and against the default 8 points per thread
    to FP32 rounding; TL rows and transform counts identical in number."""
    for N, f, steps in [(1023, 120.0, 40), (4095, 50.0, 12), (255, 30.0, 40)]:
        s = inputs.munk(N=N, freq=f, dr=25.0, steps=steps, pade_order=6)
        out = {}
        for shape in (8, ppt):
            pl = sssp.plan_for(s, tl_every=4)
            pl.set_kernel("cta")
            pl.set_shape(shape)
            assert pl.shape == shape
            pl.march(steps)
            out[shape] = (pl.read_field(), pl.read_tl()[0], pl.transform_count())
            pl.close()
        ref = _oracle(s, tl_every=4)
        _compare(out[ppt][0], out[ppt][1], ref)
        u8, u = out[8][0], out[ppt][0]
        assert np.linalg.norm(u - u8) / np.linalg.norm(u8) < 2e-5, (N, ppt)
        assert out[8][2] == out[ppt][2], (N, out[8][2], out[ppt][2])


@pytest.mark.parametrize("N", [7, 15, 31, 63, 127, 255, 511])
def test_cta_march_small_grids_against_oracle(sssp, N):
    """The one-CTA march on every small grid (each L = N + 1 takes its own pass chain: register
    twiddles and operands for L <= 1024, a fused final radix-2 pass where the chain ends with
    one), a Munk march of 30 steps against the oracle's product form.  The source sits on the
    grid point nearest 1000 m: on the coarsest grids (625 m spacing at N = 7) a Gaussian of width
    1/k0 ~ 12 m centred between points underflows FP32 at every grid point."""
    dz = 5000.0 / (N + 1)
    s = inputs.munk(N=N, freq=20.0, dr=25.0, steps=30, pade_order=4, zs=round(1000.0 / dz) * dz)
    u, tl, _, _ = _gpu(sssp, s, tl_every=3, kernel="cta")
    _compare(u, tl, _oracle(s, tl_every=3))


def test_shape_rejected_where_unsupported(sssp):
    pl = sssp.Plan(65535, 5000.0, 0.2, 25.0, 4)
    with pytest.raises(sssp.PEError):
        pl.set_shape(4)
    pl.close()
    pl = sssp.Plan(127, 5000.0, 0.2, 25.0, 4)
    with pytest.raises(sssp.PEError):
        pl.set_shape(16)  # N + 1 below 256
    pl.set_shape(8)
    pl.close()


def test_batch_autotune_restores_state_and_picks_the_fastest(sssp):
    """pe_march_batch_autotune over a batch of 64 Munk solves (N = 1023): every shape is timed,
    the fastest is set on every plan, the march's state and TL bookkeeping are restored (the
    tuned batch then gives the oracle's result), and the untimed cluster shape reports -1."""
    solves = inputs.munk_batch(count=64, steps=30)
    plans = [sssp.plan_for(s, tl_every=10) for s in solves]
    res = sssp.autotune_batch(plans, steps=6)
    ms = res["ms"]
    assert all(ms[k] is None for k in ms if k.startswith("cluster"))
    timed = {k: v for k, v in ms.items() if v is not None}
    assert set(timed) == {"cta4", "cta8", "cta16"}
    assert res["chosen"] == min(timed, key=timed.get)
    want = int(res["chosen"][3:])
    assert all(p.shape == want for p in plans)
    assert all(p.range() == (0.0, 0) for p in plans)
    sssp.march_batch(plans, 30)
    for idx in (0, 17):
        u = plans[idx].read_field()
        tl, _ = plans[idx].read_tl()
        assert tl.shape[0] == 3
        _compare(u, tl, _oracle(solves[idx], tl_every=10))
    # the tuned plans carry measured costs and launch in cost order; an untuned batch at the same
    # shape launches in call order: the same bits
    plain = [sssp.plan_for(s, tl_every=10) for s in solves]
    for p in plain:
        p.set_shape(want)
    sssp.march_batch(plain, 30)
    for a, b in zip(plans, plain):
        assert np.array_equal(a.read_field(), b.read_field())
    for p in plans + plain:
        p.close()


def test_cluster_shapes_match_oracle_and_autotune(sssp):
    """The cluster kernel's shapes on N = 8191 (8 and 16 CTAs per cluster, the transform's exchange
    pulled by remote loads or pushed by remote stores) each march the Munk case to the oracle's
    result; the exchange mode moves the same values, so pull and push give the same bits.  The
    batch autotuner then times every shape four such solves can take (the one-CTA large-grid
    kernel and the four cluster shapes), sets the fastest, restores the march, and the tuned
    batch still gives the oracle's result."""
    s = inputs.munk(N=8191, freq=100.0, dr=25.0, steps=8)
    ref = _oracle(s)
    pl = sssp.plan_for(s, tl_every=1)
    assert pl.cluster_shape == (8, 0)  # the default of N + 1 = 8192
    pl.close()
    out = {}
    for n, u in [(8, 0), (8, 1), (16, 0), (16, 1)]:
        pl = sssp.plan_for(s, tl_every=1)
        pl.set_kernel("cluster")
        pl.set_cluster_shape(n, u)
        assert pl.cluster_shape == (n, u)
        pl.march(s.steps)
        f = pl.read_field()
        tl, _ = pl.read_tl()
        pl.close()
        _compare(f, tl, ref)
        out[(n, u)] = f
    assert np.array_equal(out[(8, 0)], out[(8, 1)])
    assert np.array_equal(out[(16, 0)], out[(16, 1)])
    solves = [s] + [inputs.munk(N=8191, freq=f, dr=25.0, steps=8) for f in (120.0, 150.0, 200.0)]
    plans = [sssp.plan_for(x, tl_every=1) for x in solves]
    res = sssp.autotune_batch(plans, steps=2)
    timed = {k: v for k, v in res["ms"].items() if v is not None}
    assert set(timed) == {"cta8", "cluster8_pull", "cluster8_push", "cluster16_pull", "cluster16_push"}, timed
    assert res["chosen"] == min(timed, key=timed.get)
    want = {"cluster8_pull": (8, 0), "cluster8_push": (8, 1), "cluster16_pull": (16, 0),
            "cluster16_push": (16, 1)}.get(res["chosen"])
    for p in plans:
        assert p.range() == (0.0, 0)
        assert p.kernel == ("cluster" if want else "cta")
        if want:
            assert p.cluster_shape == want
    sssp.march_batch(plans, s.steps)
    f = plans[0].read_field()
    tl, _ = plans[0].read_tl()
    _compare(f, tl, ref)
    for p in plans:
        p.close()
    small = sssp.Plan(4095, 5000.0, 0.2, 25.0, 4)
    with pytest.raises(sssp.PEError):
        small.set_cluster_shape(16, 1)  # 16-CTA clusters from N + 1 = 8192 on
    small.set_cluster_shape(8, 1)
    assert small.cluster_shape == (8, 1)
    small.close()
    big = sssp.Plan(32767, 5000.0, 0.2, 25.0, 4)
    assert big.cluster_shape == (16, 0)
    with pytest.raises(sssp.PEError):
        big.set_cluster_shape(8, 0)  # 8-CTA rows of N + 1 = 32768 do not fit in shared memory
    big.close()
    tiny = sssp.Plan(1023, 5000.0, 0.2, 25.0, 4)
    with pytest.raises(sssp.PEError):
        tiny.set_cluster_shape(0, 0)
    assert tiny.cluster_shape == (0, -1)
    tiny.close()


# ----------------------------------------------------------------------------- FD-SSP (Section 4.3)
def _fd_oracle(s, tl_every):
    g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr)
    return O.fd_march(s.u0, s.profiles, g, s.pade_order, s.steps, r0=s.r0, tl_every=tl_every)


@pytest.mark.parametrize("N,f,p", [(255, 30.0, 4), (511, 45.0, 6), (127, 20.0, 8), (4095, 60.0, 4)])
def test_fdssp_matches_oracle(sssp, N, f, p):
    """The FD-SSP plan (3-point stencil, tridiagonal stage solves by two block scans) against the
    oracle's banded-solve FD-SSP march: field <= 1e-4, TL <= 0.1 dB."""
    s = inputs.munk(N=N, freq=f, dr=50.0, steps=200, pade_order=p)
    pl = sssp.plan_for(s, tl_every=20, op="fd3")
    pl.march(s.steps)
    u = pl.read_field()
    tl, _ = pl.read_tl()
    pl.close()
    _compare(u, tl, _fd_oracle(s, 20))


def test_fdssp_single_mode_and_norm(sssp):
    """Isovelocity (n^2 = 1) FD-SSP on a single discrete sine mode is (e^{i sigma} R(lambda_FD))^n
    times the mode (R from the library's own FP64 Pade data); over 2000 Munk steps the norm is
    conserved."""
    N, H, f, dr, steps, m = 255, 100.0, 100.0, 5.0, 300, 7
    s = inputs.isovelocity(N=N, H=H, freq=f, dr=dr, steps=steps, pade_order=4)
    n = np.arange(1, N + 1)
    s.u0 = np.sin(np.pi * m * n / (N + 1)).astype(np.complex128)
    pl = sssp.plan_for(s, op="fd3")
    pl.march(steps)
    u = pl.read_field()
    pl.close()
    g = O.Grid(N=N, H=H, k0=s.k0, dr=dr)
    plan = O.pade_plan(g.sigma, 4)
    lam = O.fd_lambdas(N, H, s.k0)[m - 1]
    expect = (np.exp(1j * g.sigma) * plan.rational(lam)) ** steps * s.u0
    assert np.linalg.norm(u - expect) / np.linalg.norm(expect) < 1e-5
    s2 = inputs.munk(N=1023, freq=50.0, dr=25.0, steps=2000, pade_order=6)
    pl = sssp.plan_for(s2, op="fd3")
    pl.march(s2.steps)
    u2 = pl.read_field()
    pl.close()
    assert abs(np.linalg.norm(u2) / np.linalg.norm(s2.u0) - 1) < 1e-4


def test_coarse_grid_sssp_converges_where_fdssp_does_not(sssp):
    """Section 4.3's coarse-grid claim, reproduced qualitatively: Munk, H = 4 km, 20 Hz, a
    reference SSSP march on 2047 points; on 127 points (31.25 m, ~2.4 points per wavelength) the
    SSSP field at the common depths is closer to the reference than FD-SSP's even on 511 points,
    and FD-SSP's error shrinks as its grid is refined.  The starter is a smooth beam
    exp(-((z - zs)/200 m)^2), resolved on every grid, so the differences are the depth
    operators' own."""
    H, f, dr, steps, zs = 4000.0, 20.0, 50.0, 400, 1000.0

    def run(N, op):
        s = inputs.munk(N=N, H=H, freq=f, dr=dr, steps=steps, pade_order=4, zs=zs)
        s.u0 = np.exp(-((s.z - zs) / 200.0) ** 2).astype(np.complex128)
        pl = sssp.plan_for(s, op=op)
        pl.march(steps)
        u = pl.read_field()
        pl.close()
        return u

    ref = run(2047, "spectral")
    err = {}
    for N, op in [(127, "spectral"), (127, "fd3"), (255, "fd3"), (511, "fd3")]:
        u = run(N, op)
        stride = 2048 // (N + 1)
        r = ref[stride - 1::stride]  # the fine grid's points at the coarse depths
        err[(N, op)] = float(np.linalg.norm(u - r) / np.linalg.norm(r))
    print("coarse-grid errors vs SSSP N=2047:", err)
    assert err[(127, "spectral")] < err[(511, "fd3")] < err[(255, "fd3")] < err[(127, "fd3")]


def test_fdssp_range_dependent_nodes(sssp):
    """FD-SSP with a range-dependent profile (Munk + eddy, a node every 2.5 km, each node's
    Thomas factors computed at set-up) against the oracle's FD-SSP march with the same nodes
    and the midpoint rule."""
    N, H, f, dr, steps = 511, 5000.0, 40.0, 50.0, 300
    s = inputs.munk(N=N, H=H, freq=f, dr=dr, steps=steps, pade_order=5)
    z = s.z
    cm = inputs.munk_c(z)
    s.profiles = [(r, inputs.n2_from_c(cm + inputs.gaussian_eddy_dc(r + 1250.0, z, -20.0, r0=7500.0, Lr=4000.0),
                                       s.c0)) for r in np.arange(0.0, steps * dr, 2500.0)]
    pl = sssp.plan_for(s, tl_every=25, op="fd3")
    pl.march(steps)
    u = pl.read_field()
    tl, _ = pl.read_tl()
    pl.close()
    _compare(u, tl, _fd_oracle(s, 25))
