// Internal interface of the cluster march (one solve spread over a thread-block cluster;
// march_cluster.cuh), used by the plan code.  Dirichlet grids with L = N + 1 in [4096, 32768].
#pragma once
#include <cuda_runtime.h>

namespace sssp {
struct SolveDesc;
}

namespace sssp_cluster {

constexpr int kMinLog2 = 12;
constexpr int kMaxLog2 = 15;

bool supported(int log2L);
// The default shape of a size: CTAs per cluster (one solve) and whether the transform's
// all-to-all exchange is pushed by remote stores (else pulled by remote loads)
int ncta(int log2L);
bool push_default(int log2L);
// Whether a shape is built for a size: ncta 0 (the default) or the default NCTA with either
// exchange (push: 1 push, 0 pull, -1 the default), and 16-CTA clusters for L = 8192, 16384.
// Every shape computes the same step; the exchange mode does not change the arithmetic
// (bitwise the same results), the cluster size changes how the transform is split (FP32
// rounding differs).
bool shape_supported(int log2L, int ncta, int push);
// how many clusters of this shape the device can hold at once (0: the shape does not fit)
cudaError_t max_active_clusters(int log2L, bool cplx, int* clusters, int ncta = 0, int push = -1);
cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, int device,
                         int ncta = 0, int push = -1);
// out[b] = scale * DST-I(in[b]) for count fields (default shape); in: N = L - 1 values per field,
// out: L values
cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, int count, long long in_stride,
                       long long out_stride, cudaStream_t st, int device);

}  // namespace sssp_cluster
