"""Python binding of the SSSP C ABI (include/sssp.h): argument marshalling only.

Every step of the march runs in the CUDA library ``_build/libsssp.so``; this module only
converts arguments (numpy arrays for host memory, torch CUDA tensors for device memory,
torch streams for ordering) and raises ``PEError`` on a non-zero status.  There is no CPU
fallback: if the library is missing the import of a plan fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

PE_OK = 0
PE_ERR_ARG = 1
PE_ERR_CUDA = 2
PE_ERR_OOM = 3
PE_ERR_NEUMANN_DIVERGED = 4
PE_ERR_TIMEOUT = 5
PE_ERR_STATE = 6
PE_ERR_NUMERIC = 7

_STATUS_NAMES = {0: "PE_OK", 1: "PE_ERR_ARG", 2: "PE_ERR_CUDA", 3: "PE_ERR_OOM", 4: "PE_ERR_NEUMANN_DIVERGED",
                 5: "PE_ERR_TIMEOUT", 6: "PE_ERR_STATE", 7: "PE_ERR_NUMERIC"}


class PEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_LIB = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sz = ctypes.c_size_t

_SIGNATURES = {
    "pe_abi_version": (_i, []),
    "pe_create_error": (ctypes.c_char_p, []),
    "pe_last_error": (ctypes.c_char_p, [_vp]),
    "pe_plan_create": (_i, [ctypes.POINTER(_vp), _i, _d, _d, _d, _i, _i, _d, _vp]),
    "pe_plan_create_bc": (_i, [ctypes.POINTER(_vp), _i, _d, _d, _d, _i, _i, _d, _i, _vp]),
    "pe_plan_destroy": (None, [_vp]),
    "pe_set_output": (_i, [_vp, _i]),
    "pe_set_field": (_i, [_vp, _vp, _i, _d]),
    "pe_set_profile": (_i, [_vp, _vp, _i, _d, _i]),
    "pe_set_profiles": (_i, [_vp, _vp, _vp, _i, _i]),
    "pe_clear_profiles": (_i, [_vp]),
    "pe_march": (_i, [_vp, _i]),
    "pe_march_batch": (_i, [ctypes.POINTER(_vp), _i, _i]),
    "pe_sync": (_i, [_vp]),
    "pe_read_field": (_i, [_vp, _vp, _i]),
    "pe_read_TL": (_i, [_vp, _vp, _sz, _vp, ctypes.POINTER(_sz)]),
    "pe_get_transform_count": (_i, [_vp, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pe_dst1": (_i, [_vp, _vp, _vp, _i]),
    "pe_dst1_noalloc": (_i, [_vp, _vp, _i, _vp]),
    "pe_dst1_batch": (_i, [_vp, _vp, _vp, _i]),
    "pe_get_range": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong)]),
    "pe_pade_coefficients": (_i, [_d, _i, _vp, _vp, _vp]),
    "pe_march_batch_steps": (_i, [ctypes.POINTER(_vp), _vp, _i]),
    "pe_plan_set_kernel": (_i, [_vp, _i]),
    "pe_plan_get_kernel": (_i, [_vp, ctypes.POINTER(_i)]),
    "pe_plan_autotune": (_i, [_vp, _i, _vp, ctypes.POINTER(_i)]),
    "pe_plan_set_shape": (_i, [_vp, _i]),
    "pe_plan_set_operator": (_i, [_vp, _i]),
    "pe_plan_get_shape": (_i, [_vp, ctypes.POINTER(_i)]),
    "pe_plan_set_cluster_shape": (_i, [_vp, _i, _i]),
    "pe_plan_get_cluster_shape": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pe_plan_autotune_shapes": (_i, [_vp, _i, _vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pe_march_batch_autotune": (_i, [ctypes.POINTER(_vp), _i, _i, _vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pe_state_size": (_sz, [_vp]),
    "pe_save_state": (_i, [_vp, _vp, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong)]),
    "pe_load_state": (_i, [_vp, _vp, _d, ctypes.c_longlong]),
    "pe_neumann_bound": (_i, [_vp, _i, _vp]),
    "pe_inject_status": (_i, [_vp, _i]),
    "pe_server_cancel": (_i, [_vp, ctypes.c_ulonglong]),
    "pe_gemm_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i]),
    "pe_gemm_batch_march": (_i, [_vp, _i]),
    "pe_gemm_batch_read_field": (_i, [_vp, _i, _vp]),
    "pe_gemm_batch_error": (ctypes.c_char_p, [_vp]),
    "pe_gemm_batch_destroy": (None, [_vp]),
    "pe_plan_bytes_estimate": (_sz, [_i, _i, _i, ctypes.c_longlong]),
    "pe_server_create": (_i, [ctypes.POINTER(_vp), _sz, _i, _i, _vp]),
    "pe_server_set_pacing": (_i, [_vp, _i]),
    "pe_server_destroy": (None, [_vp]),
    "pe_server_error": (ctypes.c_char_p, [_vp]),
    "pe_server_submit": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pe_server_step": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "pe_server_state": (_i, [_vp, ctypes.c_ulonglong, ctypes.POINTER(_i)]),
    "pe_server_take": (_i, [_vp, ctypes.c_ulonglong, _vp, _vp, _sz, ctypes.POINTER(_sz)]),
    "pe_server_stats": (_i, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz), ctypes.POINTER(_i)]),
    "pe_server_request_params": (_i, [_vp, ctypes.c_ulonglong, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                      ctypes.POINTER(_i)]),
    "pe_neumann_radius_estimate": (_i, [_vp, _i, _d, _d, _d, _d, ctypes.POINTER(_d)]),
}


class PERequest(ctypes.Structure):
    """Mirror of ``pe_request`` (include/sssp.h)."""
    _fields_ = [("N", _i), ("H", _d), ("k0", _d), ("dr", _d), ("pade_order", _i), ("neumann_terms", _i),
                ("neumann_tol", _d), ("steps", ctypes.c_longlong), ("tl_every", _i), ("u0", _vp), ("n2", _vp),
                ("node_r", _vp), ("nodes", _i), ("r0", _d), ("flags", _i)]


ADMIT_MINIMAX_C0 = 1
ADMIT_CONVERGENT_ORDER = 2


def neumann_radius_estimate(V, H: float, k0: float, b: complex) -> float:
    """Host FP64 power-iteration estimate of the spectral radius of -b L^{-1} V (the serving
    admission's convergence check; pe_neumann_radius_estimate)."""
    v = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
    rho = _d(0)
    _check(lib().pe_neumann_radius_estimate(v.ctypes.data, int(v.size), float(H), float(k0), float(b.real),
                                            float(b.imag), ctypes.byref(rho)))
    return rho.value


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsssp.so (built in-tree by ``build()``); raises if it is missing."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, plan_ptr=None):
    if status != PE_OK:
        L = lib()
        msg = L.pe_last_error(plan_ptr).decode() if plan_ptr else L.pe_create_error().decode()
        raise PEError(status, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _host_c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex64))


def pade_coefficients(sigma: float, p: int):
    """Host FP64 Pade data of the library: (b, a, d0, d) as complex128 arrays."""
    b = np.zeros(2 * p)
    a = np.zeros(2 * p)
    d = np.zeros(2 * p + 2)
    _check(lib().pe_pade_coefficients(float(sigma), int(p), b.ctypes.data, a.ctypes.data, d.ctypes.data))
    return (b[0::2] + 1j * b[1::2], a[0::2] + 1j * a[1::2], complex(d[0], d[1]), d[2::2] + 1j * d[3::2])


class Plan:
    """One range-march problem on the GPU (pe_plan)."""

    BCS = {"dirichlet": 0, "periodic": 1, "neumann": 2}

    def __init__(self, N: int, H: float, k0: float, dr: float, pade_order: int, neumann_terms: int = 0,
                 neumann_tol: float = 1e-10, stream=None, bc: str = "dirichlet"):
        L = lib()
        ptr = _vp()
        s = _stream_ptr(stream)
        _check(L.pe_plan_create_bc(ctypes.byref(ptr), int(N), float(H), float(k0), float(dr), int(pade_order),
                                   int(neumann_terms), float(neumann_tol), self.BCS[bc], s))
        self.bc = bc
        self._p = ptr
        self.N = int(N)
        self.H, self.k0, self.dr = float(H), float(k0), float(dr)
        self.pade_order, self.neumann_terms = int(pade_order), int(neumann_terms)

    # -------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            lib().pe_plan_destroy(self._p)
            self._p = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._p

    def _c(self, status):
        _check(status, self._p)

    # -------------------------------------------------------------------------------
    def set_output(self, tl_every: int):
        self._c(lib().pe_set_output(self._p, int(tl_every)))

    def set_field(self, u, r: float = 0.0):
        """u: N complex values, numpy (host) or a complex64 CUDA torch tensor (device)."""
        if _is_torch(u):
            assert u.is_contiguous() and u.numel() == self.N
            self._c(lib().pe_set_field(self._p, u.data_ptr(), 1 if u.is_cuda else 0, float(r)))
        else:
            h = _host_c64(u)
            assert h.size == self.N
            self._c(lib().pe_set_field(self._p, h.ctypes.data, 0, float(r)))

    def set_profile(self, n2, range_m: float = 0.0):
        """n^2 at the N depth points (FP64: numpy float64, or a float64 CUDA tensor)."""
        if _is_torch(n2):
            import torch
            assert n2.is_cuda and n2.is_contiguous() and n2.numel() == self.N and n2.dtype == torch.float64
            self._c(lib().pe_set_profile(self._p, n2.data_ptr(), 0, float(range_m), 1))
        elif np.iscomplexobj(n2):
            # complex n^2 (absorbing layer): interleaved (re, im) doubles
            h = np.ascontiguousarray(np.asarray(n2, dtype=np.complex128))
            assert h.size == self.N
            self._c(lib().pe_set_profile(self._p, h.ctypes.data, 1, float(range_m), 0))
        else:
            h = np.ascontiguousarray(np.asarray(n2, dtype=np.float64))
            assert h.size == self.N
            self._c(lib().pe_set_profile(self._p, h.ctypes.data, 0, float(range_m), 0))

    def set_profiles(self, n2_rows, ranges):
        r = np.ascontiguousarray(np.asarray(ranges, dtype=np.float64))
        if _is_torch(n2_rows):
            import torch
            assert n2_rows.is_cuda and n2_rows.is_contiguous() and n2_rows.numel() == self.N * r.size
            assert n2_rows.dtype == torch.float64
            self._c(lib().pe_set_profiles(self._p, n2_rows.data_ptr(), r.ctypes.data, int(r.size), 1))
        else:
            h = np.ascontiguousarray(np.asarray(n2_rows, dtype=np.float64))
            assert h.size == self.N * r.size
            self._c(lib().pe_set_profiles(self._p, h.ctypes.data, r.ctypes.data, int(r.size), 0))

    def set_profile_nodes(self, nodes: Sequence[Tuple[float, np.ndarray]]):
        """Replace the profile by (range, n2) nodes."""
        self._c(lib().pe_clear_profiles(self._p))
        if any(np.iscomplexobj(n2) for _, n2 in nodes):
            for r, n2 in nodes:
                self.set_profile(np.asarray(n2, dtype=np.complex128), r)
            return
        rows = np.stack([np.asarray(n2, dtype=np.float64) for _, n2 in nodes])
        self.set_profiles(rows, [r for r, _ in nodes])

    def march(self, steps: int):
        self._c(lib().pe_march(self._p, int(steps)))

    def sync(self):
        self._c(lib().pe_sync(self._p))

    def read_field(self, out=None):
        """Field (carrier included) as a complex64 numpy array, or into a CUDA tensor ``out``."""
        if out is not None and _is_torch(out):
            assert out.is_contiguous() and out.numel() == self.N
            self._c(lib().pe_read_field(self._p, out.data_ptr(), 1 if out.is_cuda else 0))
            return out
        h = np.empty(self.N, dtype=np.complex64)
        self._c(lib().pe_read_field(self._p, h.ctypes.data, 0))
        return h

    def read_tl(self, out=None) -> Tuple[np.ndarray, np.ndarray]:
        """TL rows (rows, N) float32 and their ranges; ``out`` may be a preallocated host
        buffer (numpy or pinned torch CPU tensor) of at least rows * N floats."""
        n = _sz(0)
        if out is not None:
            ptr = out.data_ptr() if _is_torch(out) else out.ctypes.data
            cap = out.numel() if _is_torch(out) else out.size
            self._c(lib().pe_read_TL(self._p, ptr, cap, None, ctypes.byref(n)))
            return out, None
        self._c(lib().pe_read_TL(self._p, None, 0, None, ctypes.byref(n)))
        rows = n.value
        out = np.empty((rows, self.N), dtype=np.float32)
        rng = np.empty(rows, dtype=np.float64)
        if rows:
            self._c(lib().pe_read_TL(self._p, out.ctypes.data, out.size, rng.ctypes.data, ctypes.byref(n)))
        return out, rng

    def transform_count(self) -> int:
        c = ctypes.c_ulonglong(0)
        self._c(lib().pe_get_transform_count(self._p, ctypes.byref(c)))
        return int(c.value)

    def range(self) -> Tuple[float, int]:
        r = _d(0)
        s = ctypes.c_longlong(0)
        self._c(lib().pe_get_range(self._p, ctypes.byref(r), ctypes.byref(s)))
        return r.value, s.value

    def set_kernel(self, kernel: str):
        """'auto', 'cta' (one CTA per solve) or 'cluster' (one solve over a thread-block cluster)."""
        self._c(lib().pe_plan_set_kernel(self._p, KERNELS[kernel]))

    def set_operator(self, op: str):
        """'spectral' (the paper's DST-I operator, default) or 'fd3' (FD-SSP, 3-point stencil);
        before the profile and the field."""
        self._c(lib().pe_plan_set_operator(self._p, {"spectral": 0, "fd3": 1}[op]))

    def set_shape(self, points_per_thread: int):
        """Points per thread of the one-CTA kernel: 4, 8 (default) or 16."""
        self._c(lib().pe_plan_set_shape(self._p, int(points_per_thread)))

    def set_cluster_shape(self, ncta: int = 0, push: int = -1):
        """Cluster-kernel shape: CTAs per cluster (0: the size's default; 8 for N + 1 <= 16384, 16 for
        N + 1 >= 8192) and the exchange mode (1 push, 0 pull, -1 the size's default)."""
        self._c(lib().pe_plan_set_cluster_shape(self._p, int(ncta), int(push)))

    @property
    def cluster_shape(self) -> Tuple[int, int]:
        """(CTAs per cluster, push) a cluster march of this plan takes ((0, -1): no cluster kernel)."""
        n, u = _i(0), _i(0)
        self._c(lib().pe_plan_get_cluster_shape(self._p, ctypes.byref(n), ctypes.byref(u)))
        return n.value, u.value

    @property
    def shape(self) -> int:
        """Points per thread of the one-CTA kernel a march runs (0: cluster or large-grid kernel)."""
        v = _i(0)
        self._c(lib().pe_plan_get_shape(self._p, ctypes.byref(v)))
        return v.value

    @property
    def kernel(self) -> str:
        """The kernel a march of this plan runs: 'cta' or 'cluster'."""
        k = _i(0)
        self._c(lib().pe_plan_get_kernel(self._p, ctypes.byref(k)))
        return {v: n for n, v in KERNELS.items()}[k.value]

    def autotune(self, steps: int = 4, cache: bool = True) -> dict:
        """Choose this plan's kernel by timing `steps` range steps of its own march on each
        candidate (pe_plan_autotune; the march's state is restored).  The choice is cached in a
        JSON file keyed by the device and the plan's shape — $SSSP_TUNE_CACHE, else
        ~/.cache/sssp_gb300/tune.json — and a cached choice is applied without timing."""
        import json
        path = os.environ.get("SSSP_TUNE_CACHE",
                              os.path.join(os.path.expanduser("~"), ".cache", "sssp_gb300", "tune.json"))
        try:
            import torch
            dev = torch.cuda.get_device_name(torch.cuda.current_device())
        except Exception:  # noqa: BLE001 - the key only needs a stable device label
            dev = "cuda"
        key = f"{dev}|N={self.N}|bc={self.bc}|p={self.pade_order}|terms={self.neumann_terms}|steps={int(steps)}"
        data = {}
        if cache and os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            if key in data:
                self.set_kernel(data[key]["kernel"])
                return dict(data[key], cached=True)
        ms = (ctypes.c_float * 2)()
        ch = _i(0)
        self._c(lib().pe_plan_autotune(self._p, int(steps), ctypes.cast(ms, _vp), ctypes.byref(ch)))
        res = {"kernel": {v: n for n, v in KERNELS.items()}[ch.value], "ms_cta": float(ms[0]),
               "ms_cluster": float(ms[1]) if ms[1] >= 0 else None, "steps": int(steps)}
        if cache:
            os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
            data[key] = res
            with open(path, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
        return dict(res, cached=False)

    def save_state(self):
        """Bit-exact checkpoint: (spectral state, r_set, steps)."""
        st = np.empty(int(lib().pe_state_size(self._p)) // 2, dtype=np.complex64)  # 2 L values
        r = _d(0)
        n = ctypes.c_longlong(0)
        self._c(lib().pe_save_state(self._p, st.ctypes.data, ctypes.byref(r), ctypes.byref(n)))
        return st, r.value, n.value

    def load_state(self, state, r_set: float, steps: int):
        st = np.ascontiguousarray(np.asarray(state, dtype=np.complex64))
        self._c(lib().pe_load_state(self._p, st.ctypes.data, float(r_set), int(steps)))

    def neumann_bound(self, node: int = 0) -> np.ndarray:
        rho = np.zeros(self.pade_order)
        self._c(lib().pe_neumann_bound(self._p, int(node), rho.ctypes.data))
        return rho

    def inject_status(self, status: int):
        self._c(lib().pe_inject_status(self._p, int(status)))

    def dst1_batch(self, x, out):
        """count DST-I on device tensors x, out of shape (count, N), complex64."""
        assert x.is_cuda and out.is_cuda and x.shape == out.shape and x.shape[-1] == self.N
        self._c(lib().pe_dst1_batch(self._p, x.data_ptr(), out.data_ptr(), int(x.shape[0])))
        return out

    def dst1(self, x):
        """Unnormalised DST-I of N complex values on the GPU (host numpy in/out)."""
        if _is_torch(x):
            import torch
            out = torch.empty_like(x)
            self._c(lib().pe_dst1(self._p, x.data_ptr(), out.data_ptr(), 1))
            return out
        h = _host_c64(x)
        out = np.empty_like(h)
        self._c(lib().pe_dst1(self._p, h.ctypes.data, out.ctypes.data, 0))
        return out


def plan_bytes_estimate(N: int, pade_order: int, nodes: int, tl_rows: int) -> int:
    return int(lib().pe_plan_bytes_estimate(int(N), int(pade_order), int(nodes), int(tl_rows)))


class Server:
    """The continuous-batching serving loop (pe_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_live: int = 512, chunk_steps: int = 50, stream=None):
        ptr = _vp()
        st = lib().pe_server_create(ctypes.byref(ptr), int(hbm_budget_bytes), int(max_live), int(chunk_steps),
                                    _stream_ptr(stream))
        if st != PE_OK:
            raise PEError(st, "pe_server_create")
        self._s = ptr
        self._keep = {}

    def _c(self, st):
        if st != PE_OK:
            raise PEError(st, lib().pe_server_error(self._s).decode())

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            lib().pe_server_destroy(self._s)
            self._s = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pacing(self, max_weight: int):
        """Pacing limit: a cheaper request marches up to ``max_weight`` chunks per step (1: every
        request one chunk, in lockstep with the costliest)."""
        self._c(lib().pe_server_set_pacing(self._s, int(max_weight)))

    def submit(self, solve, tl_every: int = 0, steps: Optional[int] = None, admit: int = 0) -> int:
        """Queue an ``inputs.Solve``; returns the request id.  ``admit``: ADMIT_* bits."""
        u0 = _host_c64(solve.u0)
        req = PERequest(N=solve.N, H=solve.H, k0=solve.k0, dr=solve.dr, pade_order=solve.pade_order,
                        neumann_terms=solve.neumann_terms, neumann_tol=solve.neumann_tol,
                        steps=int(steps if steps is not None else solve.steps), tl_every=int(tl_every),
                        u0=u0.ctypes.data, r0=solve.r0, flags=int(admit))
        if solve.neumann_terms > 1 and len(solve.profiles) > 0:
            n2 = np.ascontiguousarray(np.stack([np.asarray(v, dtype=np.float64) for _, v in solve.profiles]))
            nr = np.ascontiguousarray(np.array([r for r, _ in solve.profiles], dtype=np.float64))
            req.n2, req.node_r, req.nodes = n2.ctypes.data, nr.ctypes.data, nr.size
        rid = ctypes.c_ulonglong(0)
        self._c(lib().pe_server_submit(self._s, ctypes.byref(req), ctypes.byref(rid)))
        self._keep[rid.value] = solve.N
        return rid.value

    def step(self):
        live, queued, done = _i(0), _i(0), _i(0)
        self._c(lib().pe_server_step(self._s, ctypes.byref(live), ctypes.byref(queued), ctypes.byref(done)))
        return live.value, queued.value, done.value

    def state(self, rid: int) -> int:
        st = _i(0)
        self._c(lib().pe_server_state(self._s, ctypes.c_ulonglong(rid), ctypes.byref(st)))
        return st.value

    def take(self, rid: int):
        N = self._keep[rid]
        rows = _sz(0)
        self._c(lib().pe_server_take(self._s, ctypes.c_ulonglong(rid), None, None, 0, ctypes.byref(rows)))
        field = np.empty(N, dtype=np.complex64)
        tl = np.empty((rows.value, N), dtype=np.float32)
        self._c(lib().pe_server_take(self._s, ctypes.c_ulonglong(rid), field.ctypes.data,
                                     tl.ctypes.data if tl.size else None, tl.size, ctypes.byref(rows)))
        del self._keep[rid]
        return field, tl

    def params(self, rid: int):
        """(k0, n2 scale, Pade order) the request marches with after admission."""
        k0, sc, p = _d(0), _d(0), _i(0)
        self._c(lib().pe_server_request_params(self._s, ctypes.c_ulonglong(rid), ctypes.byref(k0), ctypes.byref(sc),
                                               ctypes.byref(p)))
        return k0.value, sc.value, p.value

    def cancel(self, rid: int):
        self._c(lib().pe_server_cancel(self._s, ctypes.c_ulonglong(rid)))

    def stats(self):
        a, b, c = _sz(0), _sz(0), _i(0)
        self._c(lib().pe_server_stats(self._s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"bytes_in_use": a.value, "peak_bytes": b.value, "peak_live": c.value}


KERNELS = {"auto": 0, "cta": 1, "cluster": 2}

GEMM_MODES = {"fp32": 0, "tf32": 1, "3xtf32": 2, "bf16x3": 3}


class GemmBatch:
    """Lockstep batched march with the DST-I as a dense GEMM (pe_gemm_batch_*)."""

    def __init__(self, plans: List[Plan], mode: str = "3xtf32"):
        arr = (_vp * len(plans))(*[p.handle for p in plans])
        ptr = _vp()
        st = lib().pe_gemm_batch_create(ctypes.byref(ptr), arr, len(plans), GEMM_MODES[mode])
        if st != PE_OK:
            raise PEError(st, lib().pe_last_error(plans[0].handle).decode())
        self._g = ptr
        self.N = plans[0].N

    def march(self, steps: int):
        st = lib().pe_gemm_batch_march(self._g, int(steps))
        if st != PE_OK:
            raise PEError(st, lib().pe_gemm_batch_error(self._g).decode())

    def read_field(self, index: int) -> np.ndarray:
        out = np.empty(self.N, dtype=np.complex64)
        st = lib().pe_gemm_batch_read_field(self._g, int(index), out.ctypes.data)
        if st != PE_OK:
            raise PEError(st, lib().pe_gemm_batch_error(self._g).decode())
        return out

    def close(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            lib().pe_gemm_batch_destroy(self._g)
            self._g = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# the shapes the autotuners time, in the order of their timing outputs (include/sssp.h): one CTA
# at 4/8/16 points per thread; 8-CTA clusters (N + 1 = 4096 .. 16384) pulling / pushing the
# transform's exchange; 16-CTA clusters (N + 1 = 8192 .. 32768) pulling / pushing
SHAPE_NAMES = ("cta4", "cta8", "cta16", "cluster8_pull", "cluster8_push", "cluster16_pull", "cluster16_push")


def _shape_result(ms, k, p):
    t = {n: (float(ms[i]) if ms[i] >= 0 else None) for i, n in enumerate(SHAPE_NAMES)}
    timed = {n: v for n, v in t.items() if v is not None}
    chosen = min(timed, key=timed.get) if timed else None  # the library keeps the first fastest
    if chosen is not None:
        want_cluster = k.value == KERNELS["cluster"]
        assert chosen.startswith("cluster") == want_cluster and (want_cluster or chosen == f"cta{p.value}")
    return {"chosen": chosen, "ms": t}


def autotune_batch(plans: List[Plan], steps: int = 8) -> dict:
    """Time ``steps`` range steps of the batched march of ``plans`` with every shape they can take
    (one CTA per solve at 4/8/16 points per thread, one cluster per solve), restore their state,
    and set the fastest (pe_march_batch_autotune)."""
    arr = (_vp * len(plans))(*[p.handle for p in plans])
    ms = (ctypes.c_float * len(SHAPE_NAMES))()
    k, p = _i(0), _i(0)
    st = lib().pe_march_batch_autotune(arr, len(plans), int(steps), ctypes.cast(ms, _vp), ctypes.byref(k),
                                       ctypes.byref(p))
    if st != PE_OK:
        raise PEError(st, lib().pe_last_error(plans[0].handle).decode())
    return _shape_result(ms, k, p)


def march_batch_steps(plans: List[Plan], steps: Sequence[int]):
    arr = (_vp * len(plans))(*[p.handle for p in plans])
    st_arr = np.ascontiguousarray(np.asarray(steps, dtype=np.int32))
    st = lib().pe_march_batch_steps(arr, st_arr.ctypes.data, len(plans))
    if st != PE_OK:
        raise PEError(st, lib().pe_last_error(plans[0].handle).decode())


def march_batch(plans: List[Plan], steps: int):
    """March every plan ``steps`` steps with one kernel launch per grid size."""
    arr = (_vp * len(plans))(*[p.handle for p in plans])
    st = lib().pe_march_batch(arr, len(plans), int(steps))
    if st != PE_OK:
        raise PEError(st, lib().pe_last_error(plans[0].handle).decode())


def plan_for(solve, stream=None, tl_every: int = 0, op: str = "spectral") -> Plan:
    """Plan, starter field and profile nodes for an ``inputs.Solve`` description (``op``: the
    depth operator, 'spectral' or 'fd3')."""
    pl = Plan(solve.N, solve.H, solve.k0, solve.dr, solve.pade_order, solve.neumann_terms, solve.neumann_tol,
              stream=stream, bc=getattr(solve, "bc", "dirichlet"))
    pl.set_output(tl_every)
    if op != "spectral":
        pl.set_operator(op)
    if solve.neumann_terms > 1 or op != "spectral":
        pl.set_profile_nodes(solve.profiles)
    pl.set_field(solve.u0, solve.r0)
    return pl
