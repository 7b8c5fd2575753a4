// Internal interface of the one-CTA march kernel at 4 and 16 points per thread (the library's
// default shape, 8 points per thread, is launched by the plan code itself).  Dirichlet grids with
// L = N + 1 in [256, 4096]; the field and every transform in one CTA's shared memory.
#pragma once
#include <cuda_runtime.h>

namespace sssp {
struct SolveDesc;
}

namespace sssp_shapes {

constexpr int kMinLog2 = 8;
constexpr int kMaxLog2 = 12;

bool supported(int log2L, int ppt);
// dynamic shared memory of the shape (bytes), for occupancy and validation
size_t smem_bytes(int log2L, int ppt, bool cplx);
cudaError_t launch_march(int log2L, int ppt, const sssp::SolveDesc* d, int count, const float2* tw,
                         const float* sinw, cudaStream_t st, bool cplx);

}  // namespace sssp_shapes
