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
int ncta(int log2L);  // CTAs per cluster (one solve)
// how many clusters of this shape the device can hold at once (0: the shape does not fit)
cudaError_t max_active_clusters(int log2L, bool cplx, int* clusters);
cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, int device);
// out[b] = scale * DST-I(in[b]) for count fields; in: N = L - 1 values per field, out: L values
cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, int count, long long in_stride,
                       long long out_stride, cudaStream_t st, int device);

}  // namespace sssp_cluster
