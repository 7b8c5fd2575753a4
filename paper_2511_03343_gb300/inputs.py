"""Seeded synthetic inputs for the spectral split-step Pade (SSSP) marcher.

This module only *generates inputs*: sound-speed environments, refractive
index profiles n^2(z) and starter fields.  It holds none of the marcher's
arithmetic (no transforms, no Pade coefficients, no Neumann series) so that
both the FP64 oracle's tests and the CUDA path can draw the same inputs from
it without sharing any of the method.

Environments follow the paper:
  * Munk deep-ocean profile, Eq. (Munk) in Section 4.1;
  * the synoptic eddy of Eq. (Eddy) with the parameters of Table 1, and the
    Gaussian range/depth eddy used for the range-dependent workload;
  * Gaussian and Greene starters of Section 3.2 (Eq. Greene).

All random draws use numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

C0_DEFAULT = 1500.0  # reference sound speed [m/s] used for k0 = omega / c0


# ----------------------------------------------------------------------------
# grid
# ----------------------------------------------------------------------------
def depth_grid(N: int, H: float, bc: str = "dirichlet") -> np.ndarray:
    """Depth points of the grid: Dirichlet N interior points z_n = n H/(N+1), n = 1..N;
    periodic N points z_n = n H/N, n = 0..N-1; Neumann N points z_n = n H/(N-1), n = 0..N-1."""
    if bc == "periodic":
        return (H / N) * np.arange(N, dtype=np.float64)
    if bc == "neumann":
        return (H / (N - 1)) * np.arange(N, dtype=np.float64)
    dz = H / (N + 1)
    return dz * np.arange(1, N + 1, dtype=np.float64)


# ----------------------------------------------------------------------------
# sound-speed environments
# ----------------------------------------------------------------------------
def munk_c(z: np.ndarray) -> np.ndarray:
    """Munk profile, Eq. (Munk) of Section 4.1: c = 1500(1 + 0.00737(eta + e^-eta - 1)),
    eta = 2(z - 1300)/1300, in m/s."""
    eta = 2.0 * (np.asarray(z, dtype=np.float64) - 1300.0) / 1300.0
    return 1500.0 * (1.0 + 0.00737 * (eta + np.exp(-eta) - 1.0))


def gaussian_eddy_dc(r: float, z: np.ndarray, dc: float, r0: float = 50e3, Lr: float = 10e3,
                     z0: float = 700.0, Lz: float = 400.0) -> np.ndarray:
    """Gaussian eddy perturbation dc*exp(-((r-r0)/Lr)^2 - ((z-z0)/Lz)^2) [m/s] for the
    range-dependent Munk workload (a stand-in shaped like the eddy of Section 4.2)."""
    z = np.asarray(z, dtype=np.float64)
    return dc * np.exp(-((r - r0) / Lr) ** 2 - ((z - z0) / Lz) ** 2)


def paper_eddy_dc(r: float, z: np.ndarray, beta: float = 1.7125, rx: float = 32e3, ry: float = 18e3,
                  rz: float = 250.0, x0: float = 50e3, y0: float = 0.0, z0: float = 1100.0,
                  cm: float = 40.0, y: float = 0.0) -> np.ndarray:
    """Synoptic eddy of Eq. (Eddy), Section 4.2, with the Table 1 parameters as defaults.
    The propagation plane is y = 0 and the range r plays the role of x."""
    z = np.asarray(z, dtype=np.float64)
    return (-cm * math.exp(-((r - x0) ** 2) / rx ** 2) * math.exp(-((y - y0) ** 2) / ry ** 2)
            * ((z - z0) / rz) * np.exp(-beta * (z - z0) ** 2 / rz ** 2))


def n2_from_c(c: np.ndarray, c0: float = C0_DEFAULT) -> np.ndarray:
    """Squared refractive index n^2 = (c0/c)^2."""
    return (c0 / np.asarray(c, dtype=np.float64)) ** 2


# ----------------------------------------------------------------------------
# starters (Section 3.2)
# ----------------------------------------------------------------------------
def gaussian_starter(z: np.ndarray, k0: float, zs: float) -> np.ndarray:
    """Gaussian starter u0 = sqrt(k0) exp(-k0^2 (z - zs)^2 / 2) (complex128)."""
    z = np.asarray(z, dtype=np.float64)
    return (math.sqrt(k0) * np.exp(-(k0 ** 2) * (z - zs) ** 2 / 2.0)).astype(np.complex128)


def greene_starter(z: np.ndarray, k0: float, zs: float) -> np.ndarray:
    """Greene's starter, Eq. (Greene): sqrt(k0)[1.4467 - 0.4201 k0^2 (z-zs)^2]
    exp(-k0^2 (z-zs)^2 / 3.0512) (the exponent read as k0^2 (z-zs)^2)."""
    z = np.asarray(z, dtype=np.float64)
    s2 = (k0 ** 2) * (z - zs) ** 2
    return (math.sqrt(k0) * (1.4467 - 0.4201 * s2) * np.exp(-s2 / 3.0512)).astype(np.complex128)


def modal_starter(z: np.ndarray, H: float, c: np.ndarray, freq: float, zs: float, c0: float = C0_DEFAULT,
                  max_angle_deg: float = 90.0) -> np.ndarray:
    """Normal-mode starter of Section 3.2: u(r0, z) = sqrt(2 pi) sum_m Psi_m(zs) Psi_m(z) / sqrt(kappa_m)
    over the propagating modes of the Sturm-Liouville problem Psi'' + (k^2(z) - kappa^2) Psi = 0 with
    Psi(0) = Psi(H) = 0 (the printed "+ kappa^2" read as "- kappa^2"), k = 2 pi f / c(z).

    The modes come from a second-order finite-difference discretisation on the interior grid ``z``
    (a starter generator of its own, independent of the marcher's spectral operator), normalised so
    that sum_n Psi_m(z_n)^2 dz = 1; Psi_m(zs) is linearly interpolated.  Only modes whose grazing
    angle acos(kappa_m / k0) is below ``max_angle_deg`` are kept (k0 = 2 pi f / c0).
    """
    from scipy.linalg import eigh_tridiagonal
    z = np.asarray(z, dtype=np.float64)
    N = z.size
    dz = H / (N + 1)
    k2 = (2.0 * math.pi * freq / np.asarray(c, dtype=np.float64)) ** 2
    k0 = 2.0 * math.pi * freq / c0
    diag = -2.0 / dz ** 2 + k2
    off = np.full(N - 1, 1.0 / dz ** 2)
    kap2, psi = eigh_tridiagonal(diag, off)
    psi = psi / math.sqrt(dz)
    cos_max = math.cos(math.radians(max_angle_deg))
    keep = kap2 > (k0 * cos_max) ** 2 if max_angle_deg < 90.0 else kap2 > 0
    u = np.zeros(N, dtype=np.complex128)
    zz = np.concatenate([[0.0], z, [H]])
    for m in np.nonzero(keep)[0]:
        col = np.concatenate([[0.0], psi[:, m], [0.0]])
        psi_s = np.interp(zs, zz, col)
        u += psi_s * psi[:, m] / math.sqrt(math.sqrt(kap2[m]))
    return math.sqrt(2.0 * math.pi) * u


# ----------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Solve:
    """One range-march problem: grid, Pade plan parameters, starter and profile nodes.

    ``profiles`` is a list of (range_node, n2) pairs: a range step [r, r+dr] uses the
    last node whose range is <= its midpoint r + dr/2.
    """
    name: str
    N: int
    H: float
    freq: float
    dr: float
    steps: int
    pade_order: int
    neumann_terms: int
    neumann_tol: float
    zs: float
    c0: float = C0_DEFAULT
    u0: Optional[np.ndarray] = None
    profiles: List = dataclasses.field(default_factory=list)
    r0: float = 0.0
    bc: str = "dirichlet"

    @property
    def k0(self) -> float:
        return 2.0 * math.pi * self.freq / self.c0

    @property
    def z(self) -> np.ndarray:
        return depth_grid(self.N, self.H, self.bc)


def _with_starter(s: Solve) -> Solve:
    s.u0 = gaussian_starter(s.z, s.k0, s.zs)
    return s


def isovelocity(N: int = 255, H: float = 100.0, freq: float = 100.0, dr: float = 5.0, steps: int = 1000,
                pade_order: int = 4, zs: float = 50.0, bc: str = "dirichlet") -> Solve:
    """Isovelocity waveguide, n^2 = 1 (V = 0), no Neumann terms (Dirichlet unless ``bc``)."""
    s = Solve("isovelocity", N, H, freq, dr, steps, pade_order, 0, 1e-10, zs, bc=bc)
    s.profiles = [(0.0, np.ones(N))]
    return _with_starter(s)


def munk(N: int = 4095, H: float = 5000.0, freq: float = 50.0, dr: float = 50.0, steps: int = 2000,
         pade_order: int = 6, neumann_terms: int = 12, neumann_tol: float = 1e-10, zs: float = 1000.0,
         bc: str = "dirichlet") -> Solve:
    """Range-independent Munk deep-ocean guide (grid of the boundary condition ``bc``)."""
    s = Solve("munk", N, H, freq, dr, steps, pade_order, neumann_terms, neumann_tol, zs, bc=bc)
    s.profiles = [(0.0, n2_from_c(munk_c(s.z), s.c0))]
    return _with_starter(s)


def munk_eddy(N: int = 16383, H: float = 5000.0, freq: float = 250.0, dr: float = 25.0, steps: int = 4000,
              pade_order: int = 8, neumann_terms: int = 12, neumann_tol: float = 1e-10, zs: float = 1000.0,
              seed: int = 3, dc: Optional[float] = None) -> Solve:
    """Range-dependent Munk + Gaussian eddy; the profile is refreshed at every step's
    midpoint.  dc is drawn uniformly from [-25, -10] m/s with default_rng(seed)."""
    if dc is None:
        dc = float(np.random.default_rng(seed).uniform(-25.0, -10.0))
    s = Solve("munk_eddy", N, H, freq, dr, steps, pade_order, neumann_terms, neumann_tol, zs)
    z = s.z
    cm = munk_c(z)
    s.profiles = []
    for n in range(steps):
        rmid = (n + 0.5) * dr
        s.profiles.append((n * dr, n2_from_c(cm + gaussian_eddy_dc(rmid, z, dc), s.c0)))
    s.eddy_dc = dc
    return _with_starter(s)


def munk_batch(count: int = 256, N: int = 1023, H: float = 5000.0, dr: float = 25.0, steps: int = 2000,
               pade_order: int = 6, neumann_terms: int = 12, neumann_tol: float = 1e-10, zs: float = 1000.0,
               seed: int = 4, fmin: float = 50.0, fmax: float = 500.0) -> List[Solve]:
    """Batch of range-independent Munk solves with frequencies ~ U[fmin, fmax] (default_rng(seed))."""
    freqs = np.random.default_rng(seed).uniform(fmin, fmax, count)
    out = []
    for f in freqs:
        out.append(munk(N=N, H=H, freq=float(f), dr=dr, steps=steps, pade_order=pade_order,
                        neumann_terms=neumann_terms, neumann_tol=neumann_tol, zs=zs))
    return out


def serving_trace(count: int = 1000, rate: float = 200.0, seed: int = 5, budget_bytes: float = 120e9,
                  Ns=(255, 1023, 4095, 16383, 65535), dr: float = 25.0, H0: float = 5000.0):
    """Poisson arrival trace of mixed solves (times in seconds).

    Each request: N ~ U{Ns}; environment ~ U{isovelocity (H=100 m), Munk (H=5000 m),
    Munk + random Gaussian eddy}; f ~ U[25, min(1000, 0.15 (N+1) H0 / H)] Hz (keeps dz <= lambda/2);
    range ~ U[10, 200] km; Pade order ~ U{4..8}; starter depth ~ U[0.1 H, 0.9 H].
    Returns a list of dicts (parameters only: fields and profiles are built by ``build_request``).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(Ns))
        env = ["isovelocity", "munk", "munk_eddy"][int(rng.integers(0, 3))]
        H = 100.0 if env == "isovelocity" else 5000.0
        fmax = min(1000.0, 0.15 * (N + 1) * H0 / H)
        f = float(rng.uniform(25.0, fmax))
        rng_km = float(rng.uniform(10.0, 200.0))
        p = int(rng.integers(4, 9))
        zs = float(rng.uniform(0.1 * H, 0.9 * H))
        dc = float(rng.uniform(-25.0, -10.0))
        r0 = float(rng.uniform(0.0, 200e3))
        out.append(dict(id=i, t_arrival=t, N=N, env=env, H=H, freq=f, range_m=rng_km * 1e3, dr=dr,
                        steps=int(math.ceil(rng_km * 1e3 / dr)), pade_order=p, zs=zs, eddy_dc=dc,
                        eddy_r0=r0))
    return out
