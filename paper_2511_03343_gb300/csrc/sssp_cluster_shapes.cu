// The cluster march's non-default shapes (march_cluster.cuh), timed by the shape autotuner:
// the other exchange mode of every size, and 16-CTA clusters for L = 8192 and 16384.  A
// translation unit of their own so that they compile beside the default shapes.
#include "cluster_host.cuh"

namespace sssp_cluster_host {

cudaError_t march_alt(int log2L, int ncta, bool push, const sssp::SolveDesc* d, int count, cudaStream_t st,
                      bool cplx, const ClusterTables& t) {
  if (ncta == 8) {
    switch (log2L) {
      case 12: return push ? march_t<12, 8, true>(d, count, st, cplx, t) : cudaErrorInvalidValue;
      case 13: return push ? cudaErrorInvalidValue : march_t<13, 8, false>(d, count, st, cplx, t);
      case 14: return push ? cudaErrorInvalidValue : march_t<14, 8, false>(d, count, st, cplx, t);
    }
  } else if (ncta == 16) {
    switch (log2L) {
      case 13: return push ? march_t<13, 16, true>(d, count, st, cplx, t) : march_t<13, 16, false>(d, count, st, cplx, t);
      case 14: return push ? march_t<14, 16, true>(d, count, st, cplx, t) : march_t<14, 16, false>(d, count, st, cplx, t);
      case 15: return push ? cudaErrorInvalidValue : march_t<15, 16, false>(d, count, st, cplx, t);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t fits_alt(int log2L, int ncta, bool push, bool cplx, int* clusters) {
  *clusters = 0;
  if (ncta == 8) {
    switch (log2L) {
      case 12: return push ? fits_t<12, 8, true>(cplx, clusters) : cudaErrorInvalidValue;
      case 13: return push ? cudaErrorInvalidValue : fits_t<13, 8, false>(cplx, clusters);
      case 14: return push ? cudaErrorInvalidValue : fits_t<14, 8, false>(cplx, clusters);
    }
  } else if (ncta == 16) {
    switch (log2L) {
      case 13: return push ? fits_t<13, 16, true>(cplx, clusters) : fits_t<13, 16, false>(cplx, clusters);
      case 14: return push ? fits_t<14, 16, true>(cplx, clusters) : fits_t<14, 16, false>(cplx, clusters);
      case 15: return push ? cudaErrorInvalidValue : fits_t<15, 16, false>(cplx, clusters);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace sssp_cluster_host
