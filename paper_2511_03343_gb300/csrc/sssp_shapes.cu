// Instantiations and launches of the one-CTA march kernel (march_kernel.cuh) at 4 and 16 points
// per thread, Dirichlet grids L = 256 .. 4096 (kept in a translation unit of their own so the
// library's sources compile in parallel).
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <tuple>

#include "march_kernel.cuh"
#include "shape_launch.h"

namespace sssp_shapes {

namespace {

template <int LOG2L, int PPT, bool CPLX>
cudaError_t launch_t(const sssp::SolveDesc* d, int count, const float2* tw, const float* sinw, cudaStream_t st) {
  using C = sssp::Cfg<LOG2L, PPT>;
  const size_t sm = CPLX ? C::SMEM_CPLX : C::SMEM;
  static std::mutex mu;
  static std::set<int> done;  // devices whose shared-memory attribute is set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      e = cudaFuncSetAttribute(sssp::sssp_march_kernel<LOG2L, CPLX, sssp::kBcDirichlet, PPT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      if (e != cudaSuccess) return e;
      done.insert(dev);
    }
  }
  sssp::sssp_march_kernel<LOG2L, CPLX, sssp::kBcDirichlet, PPT><<<count, C::NT, sm, st>>>(d, tw, sinw);
  return cudaGetLastError();
}

template <int LOG2L, int PPT>
cudaError_t launch_c(const sssp::SolveDesc* d, int count, const float2* tw, const float* sinw, cudaStream_t st,
                     bool cplx) {
  return cplx ? launch_t<LOG2L, PPT, true>(d, count, tw, sinw, st) : launch_t<LOG2L, PPT, false>(d, count, tw, sinw, st);
}

template <int PPT>
cudaError_t launch_p(int log2L, const sssp::SolveDesc* d, int count, const float2* tw, const float* sinw,
                     cudaStream_t st, bool cplx) {
  switch (log2L) {
    case 8: return launch_c<8, PPT>(d, count, tw, sinw, st, cplx);
    case 9: return launch_c<9, PPT>(d, count, tw, sinw, st, cplx);
    case 10: return launch_c<10, PPT>(d, count, tw, sinw, st, cplx);
    case 11: return launch_c<11, PPT>(d, count, tw, sinw, st, cplx);
    case 12: return launch_c<12, PPT>(d, count, tw, sinw, st, cplx);
  }
  return cudaErrorInvalidValue;
}

template <int LOG2L, int PPT>
size_t smem_t(bool cplx) {
  return cplx ? sssp::Cfg<LOG2L, PPT>::SMEM_CPLX : sssp::Cfg<LOG2L, PPT>::SMEM;
}

template <int PPT>
size_t smem_p(int log2L, bool cplx) {
  switch (log2L) {
    case 8: return smem_t<8, PPT>(cplx);
    case 9: return smem_t<9, PPT>(cplx);
    case 10: return smem_t<10, PPT>(cplx);
    case 11: return smem_t<11, PPT>(cplx);
    case 12: return smem_t<12, PPT>(cplx);
  }
  return 0;
}

}  // namespace

bool supported(int log2L, int ppt) { return (ppt == 4 || ppt == 16) && log2L >= kMinLog2 && log2L <= kMaxLog2; }

size_t smem_bytes(int log2L, int ppt, bool cplx) {
  if (!supported(log2L, ppt)) return 0;
  return ppt == 4 ? smem_p<4>(log2L, cplx) : smem_p<16>(log2L, cplx);
}

cudaError_t launch_march(int log2L, int ppt, const sssp::SolveDesc* d, int count, const float2* tw,
                         const float* sinw, cudaStream_t st, bool cplx) {
  if (!supported(log2L, ppt)) return cudaErrorInvalidValue;
  return ppt == 4 ? launch_p<4>(log2L, d, count, tw, sinw, st, cplx) : launch_p<16>(log2L, d, count, tw, sinw, st, cplx);
}

}  // namespace sssp_shapes
