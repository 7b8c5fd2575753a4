"""FP64 CPU oracle for the spectral split-step Pade (SSSP) range marcher.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or call it.  It shares
no code with the CUDA path (no kernels, headers, tables or helpers).

Every function is a plain, slow, obviously-correct restatement of the paper
(Walsken, Ehrhardt, Petrov, "A Spectral Split-Step Pade Method for Guided Wave
Propagation"), in complex128:

* Section 2: the propagator P = exp(i h sqrt(d_z^2 + k^2)) and its [p/p] Pade
  approximation in the sum form e^{ik0h}(d0 + sum_j d_j/(1 + b_j X)), with
  X = (k^2 - k0^2 + d_z^2)/k0^2 = V + d_z^2/k0^2, V = n^2 - 1; Eq. (1dhelmholtz)
  defines w_j by (1 + b_j X) w_j = u.
* Section 3: the isovelocity inverse L_j^{-1} applied diagonally after a
  discrete trigonometric transform (Eq. inverse_isovel): the DST-I for the
  Dirichlet case of Section 3.1 (the workloads), the DFT for periodic and the
  DCT-I for homogeneous Neumann boundaries; and the Neumann series Eq. (Neumann)
  for the depth-dependent perturbation.
* Algorithm 1 (SSSP): per range step, w_j for every Pade term, then
  u_n = e^{ihk0}(d0 u_{n-1} + sum_j d_j w_j).
* Section 4.3's comparison system, FD-SSP: the same Pade product form with the 3-point finite
  difference for d_z^2 (the stencil is our choice), each (1 + b_j X) w_j = y solved directly.

The Pade coefficients are the definition of the [p/p] approximant (Baker's
linear system for the denominator, then the numerator) solved with a library
linear solve and polynomial root finder.  The DST-I is the explicit O(N^2) sine
sum.  Readings of the paper where it is silent or garbled:

* N is the number of interior depth points, dz = H/(N+1), z_n = n dz;
* the isovelocity multiplier is 1/(1 + b_j lambda_m) with the continuous
  eigenvalue lambda_m = -(pi m/(k0 H))^2 of d_z^2/k0^2 under Dirichlet BCs;
* Algorithm 1's sums run over j = 1..p plus the d0 u term;
* the Neumann series for w_j stops after term m >= 1 once
  ||t_m||_2 <= tol * ||w_j||_2 (w_j including t_m) or when ``terms`` terms
  (m = 0..terms-1) have been summed; terms <= 1 keeps only t_0 (V ignored);
* the step r -> r + dr uses the profile node in force at the step midpoint
  (the last node whose range is <= r + dr/2);
* TL = -20 log10|u| + 10 log10(r / 1 m).

Pins (tests/test_oracle_pins.py) tie each function to mathematics other than
itself: mpmath's own Pade, the exact propagator by eigendecomposition, dense
LU solves, closed-form sine modes, scipy's DST-I and norm conservation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------
# Pade approximant of f(X) = exp(i sigma (sqrt(1+X) - 1))      (Section 2)
# ----------------------------------------------------------------------------
def taylor_coeffs(sigma: float, order: int) -> np.ndarray:
    """Taylor coefficients c_0..c_order of f(X) = exp(i sigma (sqrt(1+X) - 1)) at X = 0.

    g(X) = sqrt(1+X) - 1 = sum_{k>=1} binom(1/2, k) X^k, and f = exp(h) with
    h = i sigma g obeys f' = h' f, i.e. k f_k = sum_{j=1..k} j h_j f_{k-j}.
    """
    g = np.zeros(order + 1, dtype=np.float64)
    if order >= 1:
        g[1] = 0.5
    for k in range(1, order):
        g[k + 1] = g[k] * (0.5 - k) / (k + 1)
    h = 1j * sigma * g
    f = np.zeros(order + 1, dtype=np.complex128)
    f[0] = 1.0
    for k in range(1, order + 1):
        f[k] = sum(j * h[j] * f[k - j] for j in range(1, k + 1)) / k
    return f


@dataclasses.dataclass
class PadePlan:
    """[p/p] Pade data of exp(i sigma (sqrt(1+X) - 1)).

    q, pc: ascending coefficients of Q (q[0] = 1) and P.
    b, a : Q(X) = prod_j (1 + b_j X), P(X) = P(0) prod_j (1 + a_j X).
    d0, d: sum form P/Q = d0 + sum_j d_j / (1 + b_j X).
    """
    sigma: float
    p: int
    q: np.ndarray
    pc: np.ndarray
    b: np.ndarray
    a: np.ndarray
    d0: complex
    d: np.ndarray

    def rational(self, x) -> np.ndarray:
        """P(x)/Q(x) evaluated directly from the polynomial coefficients."""
        x = np.asarray(x, dtype=np.complex128)
        return np.polyval(self.pc[::-1], x) / np.polyval(self.q[::-1], x)

    def sum_form(self, x) -> np.ndarray:
        x = np.asarray(x, dtype=np.complex128)
        out = np.full(x.shape, self.d0, dtype=np.complex128)
        for bj, dj in zip(self.b, self.d):
            out = out + dj / (1.0 + bj * x)
        return out

    def product_form(self, x) -> np.ndarray:
        x = np.asarray(x, dtype=np.complex128)
        out = np.full(x.shape, self.pc[0], dtype=np.complex128)
        for aj, bj in zip(self.a, self.b):
            out = out * (1.0 + aj * x) / (1.0 + bj * x)
        return out


def pade_plan(sigma: float, p: int) -> PadePlan:
    """[p/p] Pade approximant (Section 2; coefficients 'according to Baker').

    Q = 1 + q_1 X + .. + q_p X^p and P = p_0 + .. + p_p X^p with Q f - P = O(X^{2p+1}):
    the rows k = p+1..2p give sum_{i=1..p} q_i c_{k-i} = -c_k, then p_k = sum_{i<=k} q_i c_{k-i}.
    """
    c = taylor_coeffs(sigma, 2 * p)
    M = np.array([[c[k - i] for i in range(1, p + 1)] for k in range(p + 1, 2 * p + 1)], dtype=np.complex128)
    rhs = -c[p + 1:2 * p + 1]
    q = np.concatenate([[1.0 + 0j], np.linalg.solve(M, rhs)])
    pc = np.array([sum(q[i] * c[k - i] for i in range(0, k + 1)) for k in range(p + 1)], dtype=np.complex128)
    # Q(X) = prod (1 + b_j X): roots X_j = -1/b_j.  np.roots wants highest degree first.
    b = -1.0 / np.roots(q[::-1])
    a = -1.0 / np.roots(pc[::-1])
    d0 = pc[p] / q[p]
    d = np.empty(p, dtype=np.complex128)
    for j in range(p):
        Pval = np.polyval(pc[::-1], -1.0 / b[j])
        den = np.prod([1.0 - b[l] / b[j] for l in range(p) if l != j])
        d[j] = Pval / den
    return PadePlan(sigma=sigma, p=p, q=q, pc=pc, b=b, a=a, d0=complex(d0), d=d)


# ----------------------------------------------------------------------------
# DST-I and the isovelocity operator                        (Section 3, 3.1)
# ----------------------------------------------------------------------------
_SINE_CACHE = {}


def sine_matrix(N: int) -> np.ndarray:
    """S[m-1, n-1] = sin(pi n m / (N+1)), n, m = 1..N (argument reduced exactly mod 2(N+1))."""
    if N not in _SINE_CACHE:
        L = N + 1
        idx = np.arange(1, N + 1, dtype=np.int64)
        nm = np.outer(idx, idx) % (2 * L)
        _SINE_CACHE.clear()
        _SINE_CACHE[N] = np.sin(np.pi * nm.astype(np.float64) / L)
    return _SINE_CACHE[N]


_DST_BACKEND = {"name": "matrix"}


def set_dst_backend(name: str) -> None:
    """'matrix' (default): the explicit sine sums below.  'fft': scipy.fft.dst(type=1), a library
    routine for the same sums (its unnormalised DST-I is twice this one), for full-length runs
    of the largest grids that the explicit sums cannot finish; pinned against 'matrix'."""
    if name not in ("matrix", "fft"):
        raise ValueError(name)
    _DST_BACKEND["name"] = name


def dst1(x: np.ndarray) -> np.ndarray:
    """DST-I along axis 0: X_m = sum_{n=1..N} x_n sin(pi n m/(N+1)), by the explicit sine sum."""
    x = np.asarray(x)
    N = x.shape[0]
    if _DST_BACKEND["name"] == "fft":
        import scipy.fft
        return 0.5 * scipy.fft.dst(x, type=1, axis=0)
    if N <= 16383:
        S = sine_matrix(N)
        return S @ x.real + 1j * (S @ x.imag) if np.iscomplexobj(x) else S @ x
    # large N: rows of the sine matrix in blocks
    L = N + 1
    idx = np.arange(1, N + 1, dtype=np.int64)
    out = np.empty(x.shape, dtype=np.complex128 if np.iscomplexobj(x) else np.float64)
    for s in range(0, N, 1024):
        rows = idx[s:s + 1024]
        Sb = np.sin(np.pi * (np.outer(rows, idx) % (2 * L)).astype(np.float64) / L)
        out[s:s + 1024] = Sb @ x.real + 1j * (Sb @ x.imag) if np.iscomplexobj(x) else Sb @ x
    return out


def dst1_at(x: np.ndarray, ms) -> np.ndarray:
    """Selected DST-I outputs X_m = sum_{n=1..N} x_n sin(pi n m/(N+1)), one explicit O(N) sum per
    requested m (for grids too large for the full matrix)."""
    x = np.asarray(x)
    N = x.shape[0]
    L = N + 1
    n = np.arange(1, N + 1, dtype=np.int64)
    out = []
    for m in ms:
        out.append(np.sum(x * np.sin(np.pi * ((n * int(m)) % (2 * L)).astype(np.float64) / L)))
    return np.array(out)


def idst1(X: np.ndarray) -> np.ndarray:
    """Inverse DST-I: x = (2/(N+1)) DST-I(X)."""
    return (2.0 / (X.shape[0] + 1)) * dst1(X)


_DFT_CACHE = {}
_DCT_CACHE = {}


def dft(x: np.ndarray) -> np.ndarray:
    """DFT along axis 0 (periodic boundaries, Section 3): X_m = sum_{n=0..N-1} x_n e^{-2 pi i n m/N},
    by the explicit sum (argument reduced exactly mod N; the matrix is kept for the last N)."""
    x = np.asarray(x)
    N = x.shape[0]
    if N not in _DFT_CACHE:
        idx = np.arange(N, dtype=np.int64)
        _DFT_CACHE.clear()
        _DFT_CACHE[N] = np.exp(-2j * np.pi * (np.outer(idx, idx) % N).astype(np.float64) / N)
    return _DFT_CACHE[N] @ x


def idft(X: np.ndarray) -> np.ndarray:
    """Inverse DFT: x_n = (1/N) sum_m X_m e^{+2 pi i n m/N}."""
    return np.conj(dft(np.conj(X))) / X.shape[0]


def dct1(x: np.ndarray) -> np.ndarray:
    """DCT-I along axis 0 (homogeneous Neumann boundaries, Section 3.1), points n = 0..N-1 with
    z_0 = 0 and z_{N-1} = H: C_m = x_0/2 + (-1)^m x_{N-1}/2 + sum_{n=1..N-2} x_n cos(pi n m/(N-1))."""
    x = np.asarray(x)
    N = x.shape[0]
    if N not in _DCT_CACHE:
        K = N - 1
        idx = np.arange(N, dtype=np.int64)
        C = np.cos(np.pi * (np.outer(idx, idx) % (2 * K)).astype(np.float64) / K)
        C[:, 0] *= 0.5
        C[:, -1] *= 0.5
        _DCT_CACHE.clear()
        _DCT_CACHE[N] = C
    return _DCT_CACHE[N] @ x


def idct1(C: np.ndarray) -> np.ndarray:
    """Inverse DCT-I: x = (2/(N-1)) DCT-I(C)."""
    return (2.0 / (C.shape[0] - 1)) * dct1(C)


def lambdas(N: int, H: float, k0: float) -> np.ndarray:
    """Eigenvalues of d_z^2/k0^2 on sin(pi m z/H): lambda_m = -(pi m/(k0 H))^2, m = 1..N."""
    m = np.arange(1, N + 1, dtype=np.float64)
    return -(np.pi * m / (k0 * H)) ** 2


def lambdas_bc(N: int, H: float, k0: float, bc: str) -> np.ndarray:
    """Eigenvalues of d_z^2/k0^2 for each boundary condition of Section 3.1:
    Dirichlet sin(pi m z/H), m = 1..N; periodic e^{2 pi i l z/H} with the signed frequency
    l = m (m <= N/2) or m - N, lambda = -(2 pi l/(k0 H))^2; Neumann cos(pi m z/H), m = 0..N-1."""
    if bc == "dirichlet":
        return lambdas(N, H, k0)
    m = np.arange(N, dtype=np.float64)
    if bc == "periodic":
        l = np.where(m <= N // 2, m, m - N)
        return -(2.0 * np.pi * l / (k0 * H)) ** 2
    if bc == "neumann":
        return -(np.pi * m / (k0 * H)) ** 2
    raise ValueError(bc)


_FWD = {"dirichlet": lambda x: dst1(x), "periodic": lambda x: dft(x), "neumann": lambda x: dct1(x)}
_INV = {"dirichlet": lambda X: idst1(X), "periodic": lambda X: idft(X), "neumann": lambda X: idct1(X)}


def apply_Linv(x: np.ndarray, bj, lam: np.ndarray, bc: str = "dirichlet") -> np.ndarray:
    """L_j^{-1} x = T^{-1}[ T[x] / (1 + b_j lambda) ]   (Eq. inverse_isovel) with the transform T
    of the boundary condition (DST-I Dirichlet, DFT periodic, DCT-I Neumann).

    ``bj`` may be a scalar or a row of p values (x then has p columns)."""
    X = _FWD[bc](x)
    if X.ndim == 1:
        return _INV[bc](X / (1.0 + bj * lam))
    return _INV[bc](X / (1.0 + np.asarray(bj)[None, :] * lam[:, None]))


# ----------------------------------------------------------------------------
# Neumann series and the SSSP step                     (Eq. Neumann, Algorithm 1)
# ----------------------------------------------------------------------------
def neumann_w(u: np.ndarray, V: np.ndarray, b: np.ndarray, lam: np.ndarray, terms: int, tol: float,
              return_counts: bool = False, bc: str = "dirichlet"):
    """w_j = sum_{m=0..M} (-b_j L_j^{-1} V)^m L_j^{-1} u for every j (columns), Eq. (Neumann).

    ``u`` is one field (N,) used by every j (sum form) or a matrix (N, p) of per-j inputs.
    Term m >= 1 is t_m = -b_j L_j^{-1}(V t_{m-1}); column j stops after term m once
    ||t_m|| <= tol ||w_j||, or after ``terms`` terms in all.
    """
    b = np.asarray(b, dtype=np.complex128)
    p = b.shape[0]
    U = np.repeat(u[:, None], p, axis=1) if u.ndim == 1 else u
    t = apply_Linv(U, b, lam, bc)
    w = t.copy()
    counts = np.ones(p, dtype=np.int64)
    active = np.ones(p, dtype=bool)
    for m in range(1, max(terms, 1)):
        if not active.any():
            break
        t = -b[None, :] * apply_Linv(V[:, None] * t, b, lam, bc)
        t[:, ~active] = 0.0
        w = w + t
        counts[active] += 1
        tn = np.linalg.norm(t, axis=0)
        wn = np.linalg.norm(w, axis=0)
        active &= ~(tn <= tol * wn)
    return (w, counts) if return_counts else w


def neumann_bound(V: np.ndarray, b: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Per Pade term j, the bound rho_j = max_n |V_n| * max_m |b_j / (1 + b_j lambda_m)| on the
    2-norm of the Neumann series' operator b_j L_j^{-1} V (Eq. Neumann): the transform of the
    boundary condition is orthogonal up to scale, so ||L_j^{-1}||_2 = max_m 1/|1 + b_j lambda_m|,
    and ||V||_2 = max |V| for the diagonal V.  rho_j < 1 makes the series converge geometrically.
    Equality holds for a constant V.  For Neumann grids the DCT-I is orthogonal in the
    trapezoid-weighted norm (weight 1/2 on the two boundary points), and the bound is in that norm."""
    b = np.asarray(b, dtype=np.complex128)
    vmax = np.max(np.abs(V))
    return np.array([vmax * np.max(np.abs(bj / (1.0 + bj * lam))) for bj in b])


@dataclasses.dataclass
class Grid:
    """Depth grid: 'dirichlet' N interior points z_n = n H/(N+1), n = 1..N; 'periodic' N points
    z_n = n H/N, n = 0..N-1; 'neumann' N points z_n = n H/(N-1), n = 0..N-1 (both boundaries)."""
    N: int
    H: float
    k0: float
    dr: float
    bc: str = "dirichlet"

    @property
    def sigma(self) -> float:
        return self.k0 * self.dr

    @property
    def lam(self) -> np.ndarray:
        if self.bc == "dirichlet":
            return lambdas(self.N, self.H, self.k0)
        return lambdas_bc(self.N, self.H, self.k0, self.bc)


def step_sum(u: np.ndarray, V: np.ndarray, grid: Grid, plan: PadePlan, terms: int, tol: float,
             counts: Optional[list] = None) -> np.ndarray:
    """One SSSP range step in the paper's sum form (Algorithm 1):
    u_n = e^{i k0 dr} (d0 u + sum_j d_j w_j).  ``counts``, if given, receives the number of
    Neumann terms summed for each j (m = 0 included)."""
    w, c = neumann_w(u, V, plan.b, grid.lam, terms, tol, return_counts=True, bc=grid.bc)
    if counts is not None:
        counts.append(np.asarray(c))
    return np.exp(1j * grid.sigma) * (plan.d0 * u + w @ plan.d)


def step_product(u: np.ndarray, V: np.ndarray, grid: Grid, plan: PadePlan, terms: int, tol: float,
                 counts: Optional[list] = None) -> np.ndarray:
    """The same step in Collins' product form prod_j (1 + a_j X)(1 + b_j X)^{-1}: stage j maps
    y -> (a_j/b_j) y + (1 - a_j/b_j) w_j with (1 + b_j X) w_j = y; then u_n = e^{i k0 dr} P(0) y.
    ``counts``, if given, receives the number of Neumann terms summed in each stage."""
    y = u.astype(np.complex128)
    cs = []
    for aj, bj in zip(plan.a, plan.b):
        w, c = neumann_w(y, V, np.array([bj]), grid.lam, terms, tol, return_counts=True, bc=grid.bc)
        cs.append(int(c[0]))
        y = (aj / bj) * y + (1.0 - aj / bj) * w[:, 0]
    if counts is not None:
        counts.append(np.array(cs))
    return np.exp(1j * grid.sigma) * plan.pc[0] * y


def profile_at(profiles: Sequence[Tuple[float, np.ndarray]], r_mid: float) -> np.ndarray:
    """n^2 of the last profile node whose range is <= r_mid (the first node if none is)."""
    chosen = profiles[0][1]
    for rn, n2 in profiles:
        if rn <= r_mid:
            chosen = n2
        else:
            break
    return np.asarray(chosen)


def transmission_loss(u: np.ndarray, r: float) -> np.ndarray:
    """TL = -20 log10|u| + 10 log10(r / 1 m)  [dB]."""
    with np.errstate(divide="ignore"):
        return -20.0 * np.log10(np.abs(u)) + 10.0 * np.log10(r)


@dataclasses.dataclass
class MarchResult:
    u: np.ndarray                 # field after the last step (full field, carrier included)
    r: float                      # range of u
    tl: np.ndarray                # (records, N) TL rows
    tl_ranges: np.ndarray         # range of each TL row


def march(u0: np.ndarray, profiles, grid: Grid, pade_order: int, steps: int, terms: int, tol: float,
          r0: float = 0.0, form: str = "sum", tl_every: int = 1, plan: Optional[PadePlan] = None,
          record_steps: Optional[Sequence[int]] = None, term_counts: Optional[list] = None) -> MarchResult:
    """Algorithm 1: march u0 from range r0 over ``steps`` steps of dr.

    The step from r to r + dr uses V = n^2 - 1 of the node in force at r + dr/2.  TL is
    recorded after every ``tl_every``-th step (tl_every = 0: never); ``record_steps``
    overrides that with an explicit list of 1-based step numbers.  ``term_counts``, if given,
    receives one array per step: the Neumann terms summed for each Pade term j.
    """
    plan = plan or pade_plan(grid.sigma, pade_order)
    stepper = step_sum if form == "sum" else step_product
    u = np.asarray(u0, dtype=np.complex128).copy()
    r = r0
    tls, trs = [], []
    rec = set(record_steps) if record_steps is not None else None
    for n in range(1, steps + 1):
        V = profile_at(profiles, r + 0.5 * grid.dr) - 1.0
        if term_counts is None:
            u = stepper(u, V, grid, plan, terms if terms > 1 else 1, tol)
        else:
            u = stepper(u, V, grid, plan, terms if terms > 1 else 1, tol, counts=term_counts)
        r = r0 + n * grid.dr
        want = (n in rec) if rec is not None else (tl_every > 0 and n % tl_every == 0)
        if want:
            tls.append(transmission_loss(u, r))
            trs.append(r)
    tl = np.array(tls) if tls else np.zeros((0, u.shape[0]))
    return MarchResult(u=u, r=r, tl=tl, tl_ranges=np.array(trs))


# ----------------------------------------------------------------------------
# FD-SSP: the same Pade propagator with the standard 3-point finite difference for d_z^2
# (the comparison of Section 4.3 and the FD-SSP remark of Section 2; the stencil is our choice)
# ----------------------------------------------------------------------------
def fd_second_difference(N: int, H: float) -> np.ndarray:
    """D2 u_n = (u_{n+1} - 2 u_n + u_{n-1}) / dz^2 on the N interior points of the Dirichlet grid
    (u_0 = u_{N+1} = 0), dz = H/(N+1), as a dense matrix."""
    dz = H / (N + 1)
    D = np.diag(np.full(N, -2.0)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)
    return D / dz ** 2


def fd_lambdas(N: int, H: float, k0: float) -> np.ndarray:
    """Eigenvalues of D2/k0^2 on sin(pi m n/(N+1)): -(4/(k0 dz)^2) sin^2(pi m/(2(N+1))), m = 1..N."""
    dz = H / (N + 1)
    m = np.arange(1, N + 1, dtype=np.float64)
    return -(4.0 / (k0 * dz) ** 2) * np.sin(np.pi * m / (2.0 * (N + 1))) ** 2


def fd_step(u: np.ndarray, V: np.ndarray, grid: Grid, plan: PadePlan) -> np.ndarray:
    """One FD-SSP range step in the product form: for each j, (1 + b_j X) w_j = y by a banded
    (tridiagonal) solve, y -> (a_j/b_j) y + (1 - a_j/b_j) w_j, with X = D2/k0^2 + V; then the
    factor e^{i k0 dr} P(0)."""
    from scipy.linalg import solve_banded
    N = grid.N
    dz = grid.H / (N + 1)
    s = 1.0 / (grid.k0 * dz) ** 2
    y = np.asarray(u, dtype=np.complex128).copy()
    for aj, bj in zip(plan.a, plan.b):
        ab = np.zeros((3, N), dtype=np.complex128)
        ab[0, 1:] = bj * s                       # super-diagonal
        ab[1, :] = 1.0 + bj * (-2.0 * s + V)     # diagonal
        ab[2, :-1] = bj * s                      # sub-diagonal
        w = solve_banded((1, 1), ab, y)
        y = (aj / bj) * y + (1.0 - aj / bj) * w
    return np.exp(1j * grid.sigma) * plan.pc[0] * y


def fd_march(u0: np.ndarray, profiles, grid: Grid, pade_order: int, steps: int, r0: float = 0.0,
             tl_every: int = 1, plan: Optional[PadePlan] = None) -> MarchResult:
    """FD-SSP march of u0 over ``steps`` steps of dr (the node in force at each step's midpoint,
    TL every ``tl_every`` steps), the finite-difference counterpart of ``march``."""
    plan = plan or pade_plan(grid.sigma, pade_order)
    u = np.asarray(u0, dtype=np.complex128).copy()
    r = r0
    tls, trs = [], []
    for n in range(1, steps + 1):
        V = profile_at(profiles, r + 0.5 * grid.dr) - 1.0
        u = fd_step(u, V, grid, plan)
        r = r0 + n * grid.dr
        if tl_every > 0 and n % tl_every == 0:
            tls.append(transmission_loss(u, r))
            trs.append(r)
    tl = np.array(tls) if tls else np.zeros((0, u.shape[0]))
    return MarchResult(u=u, r=r, tl=tl, tl_ranges=np.array(trs))


# ----------------------------------------------------------------------------
# dense brute force (tiny N only)
# ----------------------------------------------------------------------------
def dense_X(grid: Grid, V: np.ndarray) -> np.ndarray:
    """X = T^{-1} diag(lambda) T + diag(V) as a dense N x N matrix (T the transform of the
    boundary condition, built by transforming the identity)."""
    if grid.bc == "dirichlet":
        S = sine_matrix(grid.N)
        Sinv = (2.0 / (grid.N + 1)) * S
        return Sinv @ np.diag(grid.lam) @ S + np.diag(np.asarray(V, dtype=np.complex128))
    I = np.eye(grid.N, dtype=np.complex128)
    T = _FWD[grid.bc](I)
    Tinv = _INV[grid.bc](I)
    return Tinv @ np.diag(grid.lam) @ T + np.diag(np.asarray(V, dtype=np.complex128))


def dense_pade_step(X: np.ndarray, plan: PadePlan, form: str = "product") -> np.ndarray:
    """e^{i sigma} times the Pade operator as a dense matrix, each (I + b_j X)^{-1} by LU."""
    N = X.shape[0]
    I = np.eye(N, dtype=np.complex128)
    if form == "product":
        Op = plan.pc[0] * I
        for aj, bj in zip(plan.a, plan.b):
            Op = (I + aj * X) @ np.linalg.solve(I + bj * X, Op)
    else:
        Op = plan.d0 * I
        for bj, dj in zip(plan.b, plan.d):
            Op = Op + dj * np.linalg.solve(I + bj * X, I)
    return np.exp(1j * plan.sigma) * Op


def exact_propagator(X: np.ndarray, sigma: float) -> np.ndarray:
    """exp(i sigma sqrt(I + X)) for Hermitian X by eigendecomposition (principal root;
    eigenvalues below -1 give evanescent, decaying factors)."""
    ev, Q = np.linalg.eigh(X)
    root = np.sqrt((1.0 + ev).astype(np.complex128))
    return (Q * np.exp(1j * sigma * root)[None, :]) @ Q.conj().T


def modal_field(u0: np.ndarray, grid: Grid, n2: np.ndarray, r: float) -> np.ndarray:
    """Normal-mode (exact one-way) field at range r for a range-independent n^2 (the reference of
    Section 4.1, Figs. 1-2): with the eigenpairs (mu_m, Psi_m) of the Hermitian X, the modes of
    d_z^2 + k^2 have kappa_m = k0 sqrt(1 + mu_m), and u(r) = sum_m <Psi_m, u0> e^{i kappa_m r} Psi_m."""
    X = dense_X(grid, np.asarray(n2) - 1.0)
    mu, Q = np.linalg.eigh(X)
    kappa = grid.k0 * np.sqrt((1.0 + mu).astype(np.complex128))
    return Q @ (np.exp(1j * kappa * r) * (Q.conj().T @ u0))
