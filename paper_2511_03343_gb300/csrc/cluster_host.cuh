// Host-side launch helpers of the cluster march (march_cluster.cuh), shared by the translation
// units that instantiate its shapes: sssp_cluster.cu (the transform tables, the dispatch, the
// 8-CTA shapes) and sssp_cluster_shapes.cu (the 16-CTA shapes).  Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include "march_cluster.cuh"

namespace sssp_cluster_host {

// per-size transform tables of a cluster shape (R = 2 NCTA residue rows of M = L/R points)
struct ClusterTables {
  float2* twM = nullptr;  // per-pass Stockham twiddles of the M-point FFT
  float2* wL = nullptr;   // R x M: w_L^{r k1}
  float2* c = nullptr;    // R x M: e^{-i pi (r + R m)/L}
  float2* wR = nullptr;   // R/2: w_R^{k2}
};

// the tables of (log2 L, NCTA) on `device`, built and uploaded on first use (sssp_cluster.cu)
cudaError_t get_cluster_tables(int device, int log2L, int ncta, ClusterTables* out);

template <class K>
inline cudaError_t prepare(K kern, size_t smem, int ncta) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess && ncta > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

inline void cluster_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, int ncta, int clusters, int threads,
                    size_t smem, cudaStream_t st) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(unsigned(ncta * clusters));
  cfg->blockDim = dim3(unsigned(threads));
  cfg->dynamicSmemBytes = smem;
  cfg->stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(ncta);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
}

template <class K, class... A>
cudaError_t launch_cluster(K kern, int ncta, int clusters, int threads, size_t smem, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  cluster_config(&cfg, at, ncta, clusters, threads, smem, st);
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int LOG2L, int NCTA, bool PUSH>
cudaError_t march_t(const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, const ClusterTables& t) {
  using C = sssp::CCfg<LOG2L, NCTA, PUSH>;
  if (cplx) {
    auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, PUSH, true>;
    cudaError_t e = prepare(k, C::SMEM_CPLX, NCTA);
    if (e != cudaSuccess) return e;
    return launch_cluster(k, NCTA, count, C::NT, C::SMEM_CPLX, st, d, (const float2*)t.twM, (const float2*)t.wL,
                          (const float2*)t.c, (const float2*)t.wR);
  }
  auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, PUSH, false>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  return launch_cluster(k, NCTA, count, C::NT, C::SMEM, st, d, (const float2*)t.twM, (const float2*)t.wL,
                        (const float2*)t.c, (const float2*)t.wR);
}

template <int LOG2L, int NCTA, bool PUSH>
cudaError_t dst_t(const float2* in, float2* out, float scale, int count, long long is, long long os, cudaStream_t st,
                  const ClusterTables& t) {
  using C = sssp::CCfg<LOG2L, NCTA, PUSH>;
  auto k = sssp::sssp_dst_cluster_kernel<LOG2L, NCTA, PUSH>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  return launch_cluster(k, NCTA, count, C::NT, C::SMEM, st, in, out, scale, (const float2*)t.twM,
                        (const float2*)t.wL, (const float2*)t.c, (const float2*)t.wR, is, os);
}

template <int LOG2L, int NCTA, bool PUSH>
cudaError_t fits_t(bool cplx, int* clusters) {
  using C = sssp::CCfg<LOG2L, NCTA, PUSH>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  if (cplx) {
    auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, PUSH, true>;
    cudaError_t e = prepare(k, C::SMEM_CPLX, NCTA);
    if (e != cudaSuccess) return e;
    cluster_config(&cfg, at, NCTA, 1, C::NT, C::SMEM_CPLX, 0);
    return cudaOccupancyMaxActiveClusters(clusters, k, &cfg);
  }
  auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, PUSH, false>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  cluster_config(&cfg, at, NCTA, 1, C::NT, C::SMEM, 0);
  return cudaOccupancyMaxActiveClusters(clusters, k, &cfg);
}


// the 8-CTA shapes (sssp_cluster.cu: L = 4096 .. 16384) and the 16-CTA shapes
// (sssp_cluster_shapes.cu: L = 8192 .. 32768), either exchange; cudaErrorInvalidValue for a shape
// not built
cudaError_t march_8(int log2L, bool push, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx,
                    const ClusterTables& t);
cudaError_t fits_8(int log2L, bool push, bool cplx, int* clusters);
cudaError_t march_16(int log2L, bool push, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx,
                     const ClusterTables& t);
cudaError_t fits_16(int log2L, bool push, bool cplx, int* clusters);

}  // namespace sssp_cluster_host
