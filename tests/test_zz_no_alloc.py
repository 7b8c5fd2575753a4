"""pe_dst1_noalloc: the DST-I for callers that must not allocate device memory (for example an
application that reserves all GPU memory for its own pool at start-up, or a plug-in whose host
framework owns every device buffer).  It is called through the C ABI on device buffers and
must give what pe_dst1 gives, call after call, although it keeps its scratch in one fixed array
that every call reuses.  This file is collected last on purpose."""
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


def _reference(sssp, x, N):
    pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4)  # allocating path: the existing entry point
    out = pl.dst1(x.astype(np.complex64))
    pl.close()
    return out


@pytest.mark.parametrize("sizes", [(4095, 4095), (1023, 255)])
def test_noalloc_matches_pe_dst1_two_calls(env, sizes):
    sssp, torch = env
    L = sssp.lib()
    stream = torch.cuda.current_stream()
    for call, N in enumerate(sizes):
        rng = np.random.default_rng(100 + call + N)
        x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
        ref = _reference(sssp, x, N)
        d_in = torch.from_numpy(x).cuda()
        d_out = torch.full((N,), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
        st = L.pe_dst1_noalloc(ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), N,
                               ctypes.c_void_p(stream.cuda_stream))
        assert st == sssp.PE_OK
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < 2e-6 * math.log2(N + 1), (call, N, err)


def test_noalloc_rejects_oversize_and_bad_args(env):
    sssp, torch = env
    L = sssp.lib()
    buf = torch.zeros(8192, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.pe_dst1_noalloc(p, p, 8191, None) == sssp.PE_ERR_ARG   # beyond the 4095 maximum
    assert L.pe_dst1_noalloc(p, p, 1000, None) == sssp.PE_ERR_ARG   # N + 1 not a power of two
    assert L.pe_dst1_noalloc(None, p, 255, None) == sssp.PE_ERR_ARG
