// The cluster march's 16-CTA shapes (march_cluster.cuh), L = 8192 .. 32768, with the transform's
// exchange pushed or pulled: a translation unit of their own so that they compile beside the
// 8-CTA shapes of sssp_cluster.cu.
#include "cluster_host.cuh"

namespace sssp_cluster_host {

cudaError_t march_16(int log2L, bool push, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx,
                     const ClusterTables& t) {
  switch (log2L) {
    case 13: return push ? march_t<13, 16, true>(d, count, st, cplx, t) : march_t<13, 16, false>(d, count, st, cplx, t);
    case 14: return push ? march_t<14, 16, true>(d, count, st, cplx, t) : march_t<14, 16, false>(d, count, st, cplx, t);
    case 15: return push ? march_t<15, 16, true>(d, count, st, cplx, t) : march_t<15, 16, false>(d, count, st, cplx, t);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fits_16(int log2L, bool push, bool cplx, int* clusters) {
  *clusters = 0;
  switch (log2L) {
    case 13: return push ? fits_t<13, 16, true>(cplx, clusters) : fits_t<13, 16, false>(cplx, clusters);
    case 14: return push ? fits_t<14, 16, true>(cplx, clusters) : fits_t<14, 16, false>(cplx, clusters);
    case 15: return push ? fits_t<15, 16, true>(cplx, clusters) : fits_t<15, 16, false>(cplx, clusters);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sssp_cluster_host
