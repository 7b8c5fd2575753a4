"""Pins for the FP64 oracle: each check ties an oracle function to mathematics other than
itself (closed forms, a library routine, brute force, an independent high-precision route).

The ``pin_*`` helpers return an error figure; the tests assert it is below a bound, and
``test_planted_mistakes_are_caught`` plants plausible mistakes in the oracle (on the CPU)
and checks that at least one pin then fails.
"""
import math

import numpy as np
import pytest

from oracle import sssp_oracle as O
from paper_2511_03343_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _grid(N=31, H=100.0, f=100.0, dr=5.0):
    return O.Grid(N=N, H=H, k0=2 * math.pi * f / 1500.0, dr=dr)


def _rng_field(N, seed=0, lowpass=None):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    if lowpass is not None:  # keep only the first `lowpass` sine modes
        U = O.dst1(u)
        U[lowpass:] = 0
        u = O.idst1(U)
    return u


# ----------------------------------------------------------------------------- DST-I
def pin_dst_scipy(N=63):
    """DST-I against scipy.fft.dst(type=1), whose definition carries a factor 2."""
    import scipy.fft
    x = _rng_field(N, 1)
    ref = scipy.fft.dst(x.real, type=1) / 2 + 1j * scipy.fft.dst(x.imag, type=1) / 2
    return np.max(np.abs(O.dst1(x) - ref)) / np.max(np.abs(ref))


def pin_dst_single_mode(N=31, m0=5):
    """DST-I of sin(pi n m0/(N+1)) is ((N+1)/2) delta_{m,m0} (discrete orthogonality)."""
    n = np.arange(1, N + 1)
    X = O.dst1(np.sin(np.pi * n * m0 / (N + 1)).astype(np.complex128))
    ref = np.zeros(N)
    ref[m0 - 1] = (N + 1) / 2
    return np.max(np.abs(X - ref))


def pin_dst_at(N=127):
    """The one-output-at-a-time sums agree with the full sine-matrix DST-I."""
    x = _rng_field(N, 11)
    ms = [1, 2, 5, 64, 126, 127]
    return np.max(np.abs(O.dst1_at(x, ms) - O.dst1(x)[np.array(ms) - 1]))


def pin_idst_roundtrip(N=63):
    x = _rng_field(N, 2)
    return np.max(np.abs(O.idst1(O.dst1(x)) - x))


def pin_spectral_second_derivative(N=63, H=100.0, k0=0.4):
    """X (V = 0) applied to u = sin^3(a z), a = pi/H, equals u''/k0^2 by calculus:
    (sin^3)'' = 6 a^2 sin cos^2 - 3 a^2 sin^3 (u is band-limited: modes 1 and 3)."""
    g = O.Grid(N=N, H=H, k0=k0, dr=1.0)
    z = inputs.depth_grid(N, H)
    a = math.pi / H
    u = np.sin(a * z) ** 3
    d2 = (6 * a * a * np.sin(a * z) * np.cos(a * z) ** 2 - 3 * a * a * np.sin(a * z) ** 3) / k0 ** 2
    Xu = O.idst1(g.lam * O.dst1(u.astype(np.complex128)))
    return np.max(np.abs(Xu - d2)) / np.max(np.abs(d2))


# ----------------------------------------------------------------------------- Pade
def _mp_pade(sigma, p, dps=50):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    f = lambda x: mpmath.exp(1j * sigma * (mpmath.sqrt(1 + x) - 1))
    c = mpmath.taylor(f, 0, 2 * p)
    P, Q = mpmath.pade(c, p, p)
    return mpmath, P, Q


def pin_pade_vs_mpmath(sigma, p):
    """P3/P8: P/Q of the oracle against mpmath's own Taylor expansion + Pade at 50 digits,
    on lambda in [-2, 0.5]; and the oracle's Taylor coefficients against mpmath.taylor."""
    mpmath, P, Q = _mp_pade(sigma, p)
    plan = O.pade_plan(sigma, p)
    xs = np.linspace(-2.0, 0.5, 41)
    ref = np.array([complex(mpmath.polyval(P[::-1], x) / mpmath.polyval(Q[::-1], x)) for x in xs])
    e_rat = np.max(np.abs(plan.rational(xs) - ref))
    e_sum = np.max(np.abs(plan.sum_form(xs) - ref))
    e_prod = np.max(np.abs(plan.product_form(xs) - ref))
    f = lambda x: mpmath.exp(1j * sigma * (mpmath.sqrt(1 + x) - 1))
    c_ref = np.array([complex(v) for v in mpmath.taylor(f, 0, 2 * p)])
    c = O.taylor_coeffs(sigma, 2 * p)
    e_tay = np.max(np.abs(c - c_ref) / np.maximum(np.abs(c_ref), 1e-300))
    return max(e_rat, e_sum, e_prod), e_tay


def pin_pade_order(sigma=2.0, p=4):
    """P3: R(x) - exp(i sigma (sqrt(1+x) - 1)) = O(x^{2p+1}) as x -> 0: halving x divides the
    error by ~2^{2p+1}."""
    plan = O.pade_plan(sigma, p)
    ex = lambda x: np.exp(1j * sigma * (np.sqrt(1 + x) - 1))
    x1, x2 = 0.2, 0.1
    e1 = abs(plan.rational(x1) - ex(x1))
    e2 = abs(plan.rational(x2) - ex(x2))
    return math.log2(e1 / e2)


# ----------------------------------------------------------------------------- operator / step
def pin_isovelocity_mode(N=31, m0=3, steps=20):
    """P4: with V = 0 a single sine mode sin(pi m0 z/H) is an eigenvector of every Pade factor;
    after n steps it is (e^{i sigma} R(lambda_m0))^n times itself, with lambda_m0 = -(pi m0/(k0 H))^2
    from calculus and R from mpmath's Pade."""
    g = _grid(N)
    mpmath, P, Q = _mp_pade(g.sigma, 4)
    lam = -(math.pi * m0 / (g.k0 * g.H)) ** 2
    G = complex(mpmath.exp(1j * g.sigma) * mpmath.polyval(P[::-1], lam) / mpmath.polyval(Q[::-1], lam))
    z = inputs.depth_grid(N, g.H)
    u0 = np.sin(math.pi * m0 * z / g.H).astype(np.complex128)
    res = O.march(u0, [(0.0, np.ones(N))], g, 4, steps, 1, 1e-10, tl_every=0)
    return np.max(np.abs(res.u - G ** steps * u0))


def pin_bruteforce_step(N=15, seed=3, form="sum"):
    """P1: one oracle step (converged Neumann) against the dense operator
    e^{i sigma} (d0 I + sum_j d_j (I + b_j X)^{-1}) built by LU on the dense X
    (sum form) or prod_j (I + a_j X)(I + b_j X)^{-1} (product form)."""
    g = _grid(N, dr=5.0)
    rng = np.random.default_rng(seed)
    V = 0.05 * rng.standard_normal(N)
    u = _rng_field(N, seed)
    plan = O.pade_plan(g.sigma, 4)
    stepper = O.step_sum if form == "sum" else O.step_product
    got = stepper(u, V, g, plan, 200, 1e-16)
    X = O.dense_X(g, V)
    ref = O.dense_pade_step(X, plan, form) @ u
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def pin_exact_propagator(N=63, seed=4):
    """P2: for a band-limited field and a weak profile the marcher agrees with the exact
    propagator exp(i sigma sqrt(I + X)) (eigendecomposition of the Hermitian X) up to the
    Pade error, which is tiny for |lambda| << 1."""
    g = _grid(N, H=100.0, f=500.0, dr=5.0)
    z = inputs.depth_grid(N, g.H)
    # smooth profile: couples sine mode m only to m +- 2 and m +- 4, so the field stays where
    # |lambda| is small and the [6/6] Pade error is negligible
    V = 0.01 * np.cos(2 * np.pi * z / g.H) + 0.005 * np.cos(4 * np.pi * z / g.H)
    u = _rng_field(N, seed, lowpass=8)
    res = O.march(u, [(0.0, V + 1.0)], g, 6, 5, 60, 1e-15, tl_every=0)
    X = O.dense_X(g, V)
    P = O.exact_propagator(X, g.sigma)
    ref = np.linalg.matrix_power(P, 5) @ u
    return np.linalg.norm(res.u - ref) / np.linalg.norm(ref)


def pin_neumann_vs_lu(N=31, seed=5):
    """P6: the Neumann series for w_j equals the dense LU solve (I + b_j X) w_j = u."""
    g = _grid(N)
    rng = np.random.default_rng(seed)
    V = 0.05 * rng.standard_normal(N)
    u = _rng_field(N, seed)
    plan = O.pade_plan(g.sigma, 4)
    w = O.neumann_w(u, V, plan.b, g.lam, 200, 1e-16)
    X = O.dense_X(g, V)
    err = 0.0
    for j, bj in enumerate(plan.b):
        ref = np.linalg.solve(np.eye(N) + bj * X, u)
        err = max(err, np.max(np.abs(w[:, j] - ref)) / np.max(np.abs(ref)))
    return err


def pin_sum_vs_product(N=31, steps=30):
    """P7: sum and product forms march to the same field."""
    g = O.Grid(N=N, H=5000.0, k0=2 * math.pi * 50 / 1500, dr=50.0)
    z = inputs.depth_grid(N, g.H)
    n2 = inputs.n2_from_c(inputs.munk_c(z))
    u0 = inputs.gaussian_starter(z, g.k0, 1000.0) + _rng_field(N, 6, lowpass=6)
    a = O.march(u0, [(0.0, n2)], g, 6, steps, 40, 1e-14, form="sum", tl_every=0)
    b = O.march(u0, [(0.0, n2)], g, 6, steps, 40, 1e-14, form="product", tl_every=0)
    return np.linalg.norm(a.u - b.u) / np.linalg.norm(b.u)


def pin_norm_conservation(N=63, steps=40):
    """P5: for real n^2 the Pade operator is unitary (a_j = conj(b_j)), so ||u|| is conserved."""
    g = O.Grid(N=N, H=5000.0, k0=2 * math.pi * 50 / 1500, dr=50.0)
    z = inputs.depth_grid(N, g.H)
    n2 = inputs.n2_from_c(inputs.munk_c(z))
    u0 = inputs.gaussian_starter(z, g.k0, 1000.0) + _rng_field(N, 7)
    res = O.march(u0, [(0.0, n2)], g, 6, steps, 40, 1e-14, tl_every=0)
    return abs(np.linalg.norm(res.u) / np.linalg.norm(u0) - 1.0)


# ============================================================================= tests
def test_dst_against_scipy():
    assert pin_dst_scipy() < 1e-13


def test_dst_single_mode():
    assert pin_dst_single_mode() < 1e-12


def test_dst_at():
    assert pin_dst_at() < 1e-11


def test_idst_roundtrip():
    assert pin_idst_roundtrip() < 1e-12


def test_spectral_second_derivative():
    assert pin_spectral_second_derivative() < 1e-12


@pytest.mark.parametrize("sigma,p,tol", [(2.094, 4, 1e-12), (10.47, 6, 1e-9), (26.18, 8, 1e-8)])
def test_pade_against_mpmath(sigma, p, tol):
    e_val, e_tay = pin_pade_vs_mpmath(sigma, p)
    assert e_val < tol
    assert e_tay < 1e-12


def test_pade_order_of_contact():
    # 2p+1 = 9 for p = 4
    assert abs(pin_pade_order() - 9.0) < 0.6


@pytest.mark.parametrize("sigma,p", [(2.094, 4), (10.47, 6), (26.18, 8)])
def test_pade_unimodular_and_conjugate(sigma, p):
    """P3: the numerator is the conjugate of the denominator, so |R(lambda)| = 1 on the real axis
    and a_j = conj(b_j)."""
    plan = O.pade_plan(sigma, p)
    lam = np.linspace(-5, 1, 301)
    assert np.max(np.abs(np.abs(plan.rational(lam)) - 1)) < 1e-8
    assert np.max(np.abs(plan.pc - np.conj(plan.q))) < 1e-8 * np.max(np.abs(plan.q))
    for bj in plan.b:
        assert np.min(np.abs(plan.a - np.conj(bj))) < 1e-7


def test_isovelocity_single_mode():
    assert pin_isovelocity_mode() < 1e-11


@pytest.mark.parametrize("form", ["sum", "product"])
def test_bruteforce_dense_step(form):
    assert pin_bruteforce_step(form=form) < 1e-11


def test_exact_propagator():
    assert pin_exact_propagator() < 1e-6


def test_neumann_equals_lu():
    assert pin_neumann_vs_lu() < 1e-12


def test_sum_equals_product():
    assert pin_sum_vs_product() < 1e-9


def test_norm_conservation():
    assert pin_norm_conservation() < 1e-9


def test_norm_decreases_with_absorption():
    """P5 variant: a complex n^2 with a positive imaginary part (absorbing layer, Section 3.1)
    makes the norm decrease."""
    N = 63
    g = O.Grid(N=N, H=5000.0, k0=2 * math.pi * 50 / 1500, dr=50.0)
    z = inputs.depth_grid(N, g.H)
    n2 = inputs.n2_from_c(inputs.munk_c(z)).astype(np.complex128)
    n2 += 1j * 0.02 * np.clip((z - 4000.0) / 1000.0, 0, None) ** 2
    u0 = _rng_field(N, 8)
    res = O.march(u0, [(0.0, n2)], g, 6, 20, 40, 1e-14, tl_every=0)
    assert np.linalg.norm(res.u) < np.linalg.norm(u0)


def test_m0_is_isovelocity():
    """P9 (Fig. 1a): keeping only the m = 0 Neumann term equals the isovelocity march (V ignored)."""
    N = 31
    g = O.Grid(N=N, H=5000.0, k0=2 * math.pi * 50 / 1500, dr=50.0)
    z = inputs.depth_grid(N, g.H)
    n2 = inputs.n2_from_c(inputs.munk_c(z))
    u0 = inputs.gaussian_starter(z, g.k0, 1000.0)
    a = O.march(u0, [(0.0, n2)], g, 6, 10, 1, 1e-10, tl_every=0)
    b = O.march(u0, [(0.0, np.ones(N))], g, 6, 10, 12, 1e-10, tl_every=0)
    assert np.max(np.abs(a.u - b.u)) < 1e-13


def test_neumann_stops_on_tolerance():
    """The stopping rule: a loose tolerance stops early, a vanishing V needs one term."""
    g = _grid(15)
    u = _rng_field(15, 9)
    plan = O.pade_plan(g.sigma, 4)
    _, c0 = O.neumann_w(u, np.zeros(15), plan.b, g.lam, 12, 1e-10, return_counts=True)
    assert np.all(c0 == 2)  # t_1 = 0 satisfies the test right after it is formed
    _, c1 = O.neumann_w(u, 0.05 * np.ones(15), plan.b, g.lam, 12, 0.5, return_counts=True)
    _, c2 = O.neumann_w(u, 0.05 * np.ones(15), plan.b, g.lam, 12, 1e-14, return_counts=True)
    assert np.all(c1 < c2) and c2.max() == 12 and np.all(c1 >= 2)


def test_profile_midpoint_rule():
    prof = [(0.0, np.full(3, 1.0)), (10.0, np.full(3, 2.0)), (20.0, np.full(3, 3.0))]
    assert O.profile_at(prof, 9.999)[0] == 1.0
    assert O.profile_at(prof, 10.0)[0] == 2.0
    assert O.profile_at(prof, 25.0)[0] == 3.0


def test_transmission_loss_closed_form():
    tl = O.transmission_loss(np.array([1.0, 0.1, 0.01j]), 10.0)
    assert np.allclose(tl, [10.0, 30.0, 50.0])


def test_munk_profile_values():
    assert abs(inputs.munk_c(np.array([1300.0]))[0] - 1500.0) < 1e-12
    # eta = -2 at the surface: 1500 (1 + 0.00737 (e^2 - 3))
    assert abs(inputs.munk_c(np.array([0.0]))[0] - 1500 * (1 + 0.00737 * (math.e ** 2 - 3))) < 1e-9
    z = np.linspace(0, 5000, 501)
    assert np.argmin(inputs.munk_c(z)) == 130


# ----------------------------------------------------------------------------- planted mistakes
_PINS = [
    ("dst_scipy", lambda: pin_dst_scipy() < 1e-13),
    ("dst_mode", lambda: pin_dst_single_mode() < 1e-12),
    ("d2", lambda: pin_spectral_second_derivative() < 1e-12),
    ("pade_mp", lambda: pin_pade_vs_mpmath(10.47, 6)[0] < 1e-9 and pin_pade_vs_mpmath(10.47, 6)[1] < 1e-12),
    ("iso_mode", lambda: pin_isovelocity_mode() < 1e-11),
    ("brute_sum", lambda: pin_bruteforce_step(form="sum") < 1e-11),
    ("brute_prod", lambda: pin_bruteforce_step(form="product") < 1e-11),
    ("exact", lambda: pin_exact_propagator() < 1e-6),
    ("neumann_lu", lambda: pin_neumann_vs_lu() < 1e-12),
    ("sum_prod", lambda: pin_sum_vs_product() < 1e-9),
]


def _all_pins_pass():
    failed = []
    for name, ok in _PINS:
        try:
            if not ok():
                failed.append(name)
        except TypeError:  # a planted mistake with the wrong signature is a bug of the test itself
            raise
        except Exception:  # a mistake may also make a pin raise
            failed.append(name)
    return failed


def test_pins_pass_unmodified():
    assert _all_pins_pass() == []


def _mut_lambda_sign(mp):
    orig = O.lambdas
    mp.setattr(O, "lambdas", lambda N, H, k0: -orig(N, H, k0))


def _mut_lambda_index(mp):
    mp.setattr(O, "lambdas", lambda N, H, k0: -(np.pi * np.arange(0, N) / (k0 * H)) ** 2)


def _mut_sine_index(mp):
    def bad(N):
        L = N + 1
        idx = np.arange(1, N + 1)
        return np.sin(np.pi * np.outer(idx, idx + 1) / L)
    O._SINE_CACHE.clear()
    mp.setattr(O, "sine_matrix", bad)


def _mut_neumann_sign(mp):
    orig = O.neumann_w

    def bad(u, V, b, lam, terms, tol, return_counts=False, bc="dirichlet"):
        return orig(u, -V, b, lam, terms, tol, return_counts, bc=bc)
    mp.setattr(O, "neumann_w", bad)


def _mut_neumann_order(mp):
    """Apply V after L^{-1} instead of before (the factors do not commute)."""
    def bad(u, V, b, lam, terms, tol, return_counts=False, bc="dirichlet"):
        b = np.asarray(b, dtype=np.complex128)
        U = np.repeat(u[:, None], len(b), axis=1) if u.ndim == 1 else u
        t = O.apply_Linv(U, b, lam, bc)
        w = t.copy()
        for m in range(1, max(terms, 1)):
            t = -b[None, :] * V[:, None] * O.apply_Linv(t, b, lam, bc)
            w = w + t
        return (w, np.full(len(b), terms)) if return_counts else w
    mp.setattr(O, "neumann_w", bad)


def _mut_drop_d0(mp):
    orig = O.pade_plan

    def bad(sigma, p):
        pl = orig(sigma, p)
        pl.d0 = 0.0
        return pl
    mp.setattr(O, "pade_plan", bad)


def _mut_taylor_term(mp):
    orig = O.taylor_coeffs

    def bad(sigma, order):
        c = orig(sigma, order).copy()
        if order >= 3:
            c[3] = 0.0
        return c
    mp.setattr(O, "taylor_coeffs", bad)


def _mut_carrier_sign(mp):
    orig = O.step_sum
    def bad(u, V, grid, plan, terms, tol, counts=None):
        return orig(u, V, grid, plan, terms, tol, counts) * np.exp(-2j * grid.sigma)
    mp.setattr(O, "step_sum", bad)


def _mut_transposed_pair(mp):
    """Swap a_j and b_j (numerator and denominator)."""
    orig = O.pade_plan

    def bad(sigma, p):
        pl = orig(sigma, p)
        pl.a, pl.b = pl.b.copy(), pl.a.copy()
        return pl
    mp.setattr(O, "pade_plan", bad)


@pytest.mark.parametrize("mutation", [_mut_lambda_sign, _mut_lambda_index, _mut_sine_index, _mut_neumann_sign,
                                      _mut_neumann_order, _mut_drop_d0, _mut_taylor_term, _mut_carrier_sign,
                                      _mut_transposed_pair])
def test_planted_mistakes_are_caught(monkeypatch, mutation):
    mutation(monkeypatch)
    try:
        failed = _all_pins_pass()
    finally:
        O._SINE_CACHE.clear()
    assert failed, f"no pin caught {mutation.__name__}"


# ----------------------------------------------------------------------------- other boundary conditions
def test_dft_and_dct_against_library():
    """DFT vs numpy.fft.fft; DCT-I vs scipy.fft.dct(type=1), whose definition carries a factor 2;
    both inverses round-trip."""
    import scipy.fft
    x = _rng_field(64, 21)
    assert np.max(np.abs(O.dft(x) - np.fft.fft(x))) < 1e-11
    ref = scipy.fft.dct(x.real, type=1) / 2 + 1j * scipy.fft.dct(x.imag, type=1) / 2
    assert np.max(np.abs(O.dct1(x) - ref)) < 1e-11
    assert np.max(np.abs(O.idft(O.dft(x)) - x)) < 1e-12
    assert np.max(np.abs(O.idct1(O.dct1(x)) - x)) < 1e-12


@pytest.mark.parametrize("bc,N,mode", [("periodic", 32, 3), ("periodic", 32, -5), ("neumann", 33, 4), ("neumann", 33, 0)])
def test_single_mode_other_bc(bc, N, mode):
    """A single eigenmode of d_z^2 under the boundary condition (e^{2 pi i l z/H} periodic,
    cos(pi m z/H) Neumann) marched in isovelocity is (e^{i sigma} R(lambda))^n times itself,
    with lambda from calculus and R from mpmath's Pade."""
    g = O.Grid(N=N, H=100.0, k0=2 * math.pi * 100 / 1500.0, dr=5.0, bc=bc)
    mpmath, P, Q = _mp_pade(g.sigma, 4)
    z = inputs.depth_grid(N, g.H, bc)
    if bc == "periodic":
        u0 = np.exp(2j * np.pi * mode * z / g.H)
        lam = -(2 * np.pi * mode / (g.k0 * g.H)) ** 2
    else:
        u0 = np.cos(np.pi * mode * z / g.H).astype(np.complex128)
        lam = -(np.pi * mode / (g.k0 * g.H)) ** 2
    G = complex(mpmath.exp(1j * g.sigma) * mpmath.polyval(P[::-1], lam) / mpmath.polyval(Q[::-1], lam))
    res = O.march(u0, [(0.0, np.ones(N))], g, 4, 15, 1, 1e-10, tl_every=0)
    assert np.max(np.abs(res.u - G ** 15 * u0)) < 1e-11


@pytest.mark.parametrize("bc,N", [("periodic", 16), ("neumann", 17)])
@pytest.mark.parametrize("form", ["sum", "product"])
def test_bruteforce_step_other_bc(bc, N, form):
    """P1 for the periodic and Neumann transforms: one step (converged Neumann series) equals
    the dense LU operator built on the dense X of that boundary condition."""
    g = O.Grid(N=N, H=100.0, k0=2 * math.pi * 100 / 1500.0, dr=5.0, bc=bc)
    rng = np.random.default_rng(31)
    V = 0.05 * rng.standard_normal(N)
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    plan = O.pade_plan(g.sigma, 4)
    stepper = O.step_sum if form == "sum" else O.step_product
    got = stepper(u, V, g, plan, 200, 1e-16)
    ref = O.dense_pade_step(O.dense_X(g, V), plan, form) @ u
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-11


def test_spectral_second_derivative_other_bc():
    """The spectral d_z^2 of each transform on a band-limited function equals calculus:
    periodic cos(2 pi z/H) + sin(6 pi z/H); Neumann cos(pi z/H) + cos(3 pi z/H)."""
    H, k0 = 100.0, 0.4
    for bc, N, f, d2 in [
        ("periodic", 64, lambda z: np.cos(2 * np.pi * z / H) + np.sin(6 * np.pi * z / H),
         lambda z: -(2 * np.pi / H) ** 2 * np.cos(2 * np.pi * z / H) - (6 * np.pi / H) ** 2 * np.sin(6 * np.pi * z / H)),
        ("neumann", 65, lambda z: np.cos(np.pi * z / H) + np.cos(3 * np.pi * z / H),
         lambda z: -(np.pi / H) ** 2 * np.cos(np.pi * z / H) - (3 * np.pi / H) ** 2 * np.cos(3 * np.pi * z / H)),
    ]:
        g = O.Grid(N=N, H=H, k0=k0, dr=1.0, bc=bc)
        z = inputs.depth_grid(N, H, bc)
        fwd = O.dft if bc == "periodic" else O.dct1
        inv = O.idft if bc == "periodic" else O.idct1
        Xu = inv(g.lam * fwd(f(z).astype(np.complex128)))
        assert np.max(np.abs(Xu - d2(z) / k0 ** 2)) / np.max(np.abs(d2(z) / k0 ** 2)) < 1e-11


@pytest.mark.parametrize("bc,N", [("periodic", 64), ("neumann", 65)])
def test_norm_conservation_other_bc(bc, N):
    """P5: the step is unitary for real n^2 — in the plain 2-norm (periodic) and in the
    trapezoid-weighted norm (Neumann: end points weighted 1/2, the DCT-I's inner product)."""
    g = O.Grid(N=N, H=5000.0, k0=2 * math.pi * 50 / 1500, dr=50.0, bc=bc)
    z = inputs.depth_grid(N, g.H, bc)
    n2 = inputs.n2_from_c(inputs.munk_c(z))
    rng = np.random.default_rng(41)
    u0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    res = O.march(u0, [(0.0, n2)], g, 6, 30, 40, 1e-14, tl_every=0)
    w = np.ones(N)
    if bc == "neumann":
        w[0] = w[-1] = 0.5
    nrm = lambda u: math.sqrt(np.sum(w * np.abs(u) ** 2))
    assert abs(nrm(res.u) / nrm(u0) - 1) < 1e-9


def test_modal_field_is_exact_propagator():
    """The normal-mode field after n steps equals the n-th power of exp(i sigma sqrt(I + X))."""
    g = O.Grid(N=31, H=100.0, k0=2 * math.pi * 100 / 1500.0, dr=5.0)
    z = inputs.depth_grid(31, g.H)
    n2 = 1.0 + 0.01 * np.cos(2 * np.pi * z / g.H)
    u0 = _rng_field(31, 51)
    P = O.exact_propagator(O.dense_X(g, n2 - 1.0), g.sigma)
    ref = np.linalg.matrix_power(P, 7) @ u0
    assert np.max(np.abs(O.modal_field(u0, g, n2, 7 * g.dr) - ref)) < 1e-12


def test_modal_starter_isovelocity_closed_form():
    """Isovelocity guide: the finite-difference modes are sin(pi m z/H) with
    kappa_m^2 = k^2 - (2/dz)^2 sin^2(pi m dz/(2H)); the starter is sqrt(2 pi) sum over them."""
    N, H, f, zs = 127, 100.0, 100.0, 37.0
    z = inputs.depth_grid(N, H)
    c = np.full(N, 1500.0)
    u = inputs.modal_starter(z, H, c, f, zs)
    dz = H / (N + 1)
    k = 2 * math.pi * f / 1500.0
    ref = np.zeros(N)
    zz = np.concatenate([[0.0], z, [H]])
    for m in range(1, N + 1):
        kap2 = k * k - (2 / dz) ** 2 * math.sin(math.pi * m * dz / (2 * H)) ** 2
        if kap2 <= 0:
            continue
        psi = np.sin(np.pi * m * z / H) * math.sqrt(2.0 / H)
        psi_s = np.interp(zs, zz, np.concatenate([[0.0], psi, [0.0]]))
        ref += psi_s * psi / kap2 ** 0.25
    ref *= math.sqrt(2 * math.pi)
    assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) < 1e-9


def _dense_neumann_operator(V, bj, grid):
    """b_j L_j^{-1} diag(V) as a dense matrix, column by column through the oracle's L^{-1}."""
    I = np.eye(grid.N)
    cols = [bj * O.apply_Linv(V * I[:, k], bj, grid.lam, grid.bc) for k in range(grid.N)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "neumann"])
def test_neumann_bound_is_the_operator_norm_for_constant_V(bc):
    # constant V: b_j L_j^{-1} V = v b_j L_j^{-1}, whose 2-norm is exactly |v| max |b/(1+b lambda)|
    N = 32 if bc != "neumann" else 33
    grid = O.Grid(N, 400.0, 2 * np.pi * 25 / 1500.0, 20.0, bc=bc)
    plan = O.pade_plan(grid.sigma, 4)
    V = np.full(N, -0.013)
    rho = O.neumann_bound(V, plan.b, grid.lam)
    # the DCT-I is orthogonal in the trapezoid-weighted norm (1/2 on both boundary points)
    w = np.ones(N)
    if bc == "neumann":
        w[0] = w[-1] = 0.5
    for j, bj in enumerate(plan.b):
        A = _dense_neumann_operator(V, bj, grid)
        nrm = np.linalg.norm(np.sqrt(w)[:, None] * A / np.sqrt(w)[None, :], 2)
        assert abs(nrm - rho[j]) <= 1e-10 * rho[j]


def test_neumann_bound_bounds_a_varying_V_and_predicts_convergence():
    grid = O.Grid(63, 500.0, 2 * np.pi * 50 / 1500.0, 25.0)
    z = inputs.depth_grid(63, 500.0)
    V = O.profile_at([(0.0, inputs.n2_from_c(inputs.munk_c(z), 1500.0))], 0.0) - 1.0
    plan = O.pade_plan(grid.sigma, 6)
    rho = O.neumann_bound(V, plan.b, grid.lam)
    for j, bj in enumerate(plan.b):
        nrm = np.linalg.norm(_dense_neumann_operator(V, bj, grid), 2)
        assert nrm <= rho[j] * (1 + 1e-12)
    # every rho_j < 1 here: the terms of each series shrink at least geometrically, so 40 terms
    # reach a relative tolerance of rho^39
    assert rho.max() < 1.0
    u = np.sin(np.pi * 3 * z / 500.0).astype(np.complex128)
    w40, counts = O.neumann_w(u, V, plan.b, grid.lam, 40, 0.0, return_counts=True)
    w80 = O.neumann_w(u, V, plan.b, grid.lam, 80, 0.0)
    err = np.linalg.norm(w40 - w80, axis=0) / np.linalg.norm(w80, axis=0)
    bound = rho ** 40 / (1 - rho) * np.linalg.norm(O.apply_Linv(np.repeat(u[:, None], 6, 1), plan.b, grid.lam), axis=0) \
        / np.linalg.norm(w80, axis=0)
    assert np.all(err <= bound * (1 + 1e-6) + 1e-15)


@pytest.mark.parametrize("N", [7, 255, 1023, 4095])
def test_fft_dst_backend_equals_the_sine_sums(N):
    """The library DST-I backend (used for full-length runs of the largest grids) gives the
    explicit sine sums, for vectors and for matrices of columns."""
    rng = np.random.default_rng(N + 3)
    x = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    ref = O.dst1(x)
    try:
        O.set_dst_backend("fft")
        got = O.dst1(x)
        got1 = O.dst1(x[:, 0])
    finally:
        O.set_dst_backend("matrix")
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale * math.log2(N + 1)
    assert np.max(np.abs(got1 - ref[:, 0])) <= 1e-12 * scale * math.log2(N + 1)
    with pytest.raises(ValueError):
        O.set_dst_backend("cuda")


@pytest.mark.parametrize("N", [16383, 65535])
def test_fft_dst_backend_at_the_largest_grids_sampled(N):
    """At the grid sizes of the stored full-length runs (N = 16383 and 65535), the library
    DST-I backend equals the explicit O(N) sine sums (dst1_at) at sampled modes: the lowest and
    highest, the middle, powers of two and random ones."""
    rng = np.random.default_rng(N + 11)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ms = sorted(set([1, 2, 3, N // 2, (N + 1) // 2, N - 1, N] + [1 << k for k in range(1, int(math.log2(N)))]
                    + list(rng.integers(1, N + 1, 24))))
    ref = O.dst1_at(x, ms)
    try:
        O.set_dst_backend("fft")
        got = O.dst1(x)[np.array(ms) - 1]
    finally:
        O.set_dst_backend("matrix")
    scale = np.sqrt(N) * np.sqrt(np.mean(np.abs(x) ** 2))
    assert np.max(np.abs(got - ref)) <= 1e-11 * scale * math.log2(N + 1)


# ----------------------------------------------------------------------------- FD-SSP (Section 4.3)
def test_fd_second_difference_eigenpairs():
    """The 3-point D2 is diagonalised by the DST-I: D2 sin(pi m n/(N+1)) equals
    -(4/dz^2) sin^2(pi m/(2(N+1))) sin(pi m n/(N+1)) (a trigonometric identity), for every m."""
    N, H = 31, 100.0
    D = O.fd_second_difference(N, H)
    k0 = 0.37
    lam = O.fd_lambdas(N, H, k0)
    n = np.arange(1, N + 1)
    for m in (1, 2, 7, 16, 31):
        v = np.sin(np.pi * m * n / (N + 1))
        assert np.max(np.abs(D @ v / k0 ** 2 - lam[m - 1] * v)) < 1e-10 * np.max(np.abs(D)) / k0 ** 2
    # and it tends to the continuous eigenvalue for m << N
    assert abs(lam[0] / O.lambdas(N, H, k0)[0] - 1) < 1e-3


def test_fd_single_mode_isovelocity_closed_form():
    """In isovelocity a single discrete sine mode marched by FD-SSP is (e^{i sigma} R(lambda_FD))^n
    times itself, R from mpmath's own Pade at the finite-difference eigenvalue."""
    N, H, k0, dr, p, steps, m = 63, 100.0, 2 * math.pi * 100 / 1500, 5.0, 4, 30, 5
    g = O.Grid(N=N, H=H, k0=k0, dr=dr)
    mpmath, P, Q = _mp_pade(g.sigma, p)
    lam = float(O.fd_lambdas(N, H, k0)[m - 1])
    R = complex(mpmath.polyval(P[::-1], lam) / mpmath.polyval(Q[::-1], lam))
    n = np.arange(1, N + 1)
    u0 = np.sin(np.pi * m * n / (N + 1)).astype(np.complex128)
    res = O.fd_march(u0, [(0.0, np.ones(N))], g, p, steps, tl_every=0)
    expect = (np.exp(1j * g.sigma) * R) ** steps * u0
    assert np.max(np.abs(res.u - expect)) < 1e-10


def test_fd_step_equals_dense_pade_operator():
    """One FD-SSP step with a Munk profile equals e^{i sigma} prod_j (I + a_j X)(I + b_j X)^{-1}
    applied by dense LU to X = D2/k0^2 + diag(V) (the banded solve is an independent route)."""
    N, H = 47, 5000.0
    z = inputs.depth_grid(N, H)
    V = inputs.n2_from_c(inputs.munk_c(z)) - 1.0
    k0 = 2 * math.pi * 30 / 1500
    g = O.Grid(N=N, H=H, k0=k0, dr=50.0)
    plan = O.pade_plan(g.sigma, 5)
    X = O.fd_second_difference(N, H) / k0 ** 2 + np.diag(V)
    u = _rng_field(N, 5)
    got = O.fd_step(u, V, g, plan)
    ref = O.dense_pade_step(X.astype(np.complex128), plan, form="product") @ u
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_fd_norm_conserved_and_converges_to_spectral():
    """FD-SSP conserves the norm for real n^2 (X real symmetric, |R| = 1 on the real axis) and,
    for a smooth field, approaches the spectral marcher as the grid is refined (second order)."""
    H, f, dr, steps = 5000.0, 30.0, 50.0, 40
    errs = []
    for N in (127, 255, 511):
        z = inputs.depth_grid(N, H)
        V = inputs.n2_from_c(inputs.munk_c(z)) - 1.0
        k0 = 2 * math.pi * f / 1500
        g = O.Grid(N=N, H=H, k0=k0, dr=dr)
        u0 = inputs.gaussian_starter(z, k0, 1000.0) * 0 + np.exp(-((z - 1200.0) / 300.0) ** 2)
        fd = O.fd_march(u0, [(0.0, V + 1.0)], g, 4, steps, tl_every=0)
        assert abs(np.linalg.norm(fd.u) / np.linalg.norm(u0) - 1) < 1e-10
        sp = O.march(u0, [(0.0, V + 1.0)], g, 4, steps, 40, 1e-13, tl_every=0, form="product")
        errs.append(np.linalg.norm(fd.u - sp.u) / np.linalg.norm(sp.u))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.0  # about 4 for a second-order stencil
