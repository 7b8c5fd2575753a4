"""pe_dst1_noalloc: the DST-I for callers that must not allocate device memory (for example an
application that reserves all GPU memory for its own pool at start-up, or a plug-in whose host
framework owns every device buffer).  It is called through the C ABI on device buffers and
must give what the FP64 oracle's explicit sine sums and pe_dst1 give, call after call, although
it keeps its scratch in one fixed array that every call reuses.  This file is collected last on
purpose."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_03343_gb300 import build
    build.build()
    from paper_2511_03343_gb300 import sssp
    return sssp, torch


def _pe_dst1(sssp, x, N):
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)  # allocating path: the existing entry point
    out = pl.dst1(x.astype(np.complex64))
    pl.close()
    return out


def _oracle_dst1(x):
    from oracle import sssp_oracle as O
    return O.dst1(x.astype(np.complex128))


def _tol(N):
    # FP32 transform of length N + 1: rounding grows like log2(N + 1)
    return 2e-6 * math.log2(N + 1)


def _call(sssp, d_in, d_out, N, stream):
    return sssp.lib().pe_dst1_noalloc(ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), N,
                                      ctypes.c_void_p(stream) if stream is not None else None)


@pytest.mark.parametrize("sizes", [(4095, 4095), (1023, 255)])
def test_noalloc_matches_oracle_and_pe_dst1_two_calls(env, sizes):
    sssp, torch = env
    stream = torch.cuda.current_stream()
    for call, N in enumerate(sizes):
        rng = np.random.default_rng(100 + call + N)
        x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
        ref = _oracle_dst1(x)
        alloc = _pe_dst1(sssp, x, N)
        d_in = torch.from_numpy(x).cuda()
        d_out = torch.full((N,), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
        assert _call(sssp, d_in, d_out, N, stream.cuda_stream) == sssp.PE_OK
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < _tol(N), (call, N, "vs oracle", err)
        err2 = np.max(np.abs(got - alloc)) / np.max(np.abs(alloc))
        assert err2 < _tol(N), (call, N, "vs pe_dst1", err2)


def test_noalloc_allocates_nothing_in_place_and_default_stream(env):
    """After a first call (the per-device set-up), a call leaves the device's free memory as it
    was; the result is right with in == out and on the legacy default stream (NULL)."""
    sssp, torch = env
    N = 2047
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    ref = _oracle_dst1(x)
    buf = torch.from_numpy(x).cuda()
    warm = torch.empty_like(buf)
    assert _call(sssp, buf, warm, N, None) == sssp.PE_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(sssp, buf, buf, N, None) == sssp.PE_OK  # in place, NULL stream
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    got = buf.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < _tol(N)


def test_noalloc_rejects_oversize_and_bad_args(env):
    sssp, torch = env
    L = sssp.lib()
    buf = torch.zeros(8192, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.pe_dst1_noalloc(p, p, 8191, None) == sssp.PE_ERR_ARG   # beyond the 4095 maximum
    assert L.pe_dst1_noalloc(p, p, 1000, None) == sssp.PE_ERR_ARG   # N + 1 not a power of two
    assert L.pe_dst1_noalloc(p, p, 2**31 - 1, None) == sssp.PE_ERR_ARG   # no overflow on huge N
    assert L.pe_dst1_noalloc(p, p, 0, None) == sssp.PE_ERR_ARG
    assert L.pe_dst1_noalloc(None, p, 255, None) == sssp.PE_ERR_ARG
