// Host side of the cluster march (march_cluster.cuh): per-size tables, launch with the
// cluster dimension, and the check that a cluster of this shape fits on the device.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "cluster_launch.h"
#include "march_cluster.cuh"

namespace {

using sssp::CCfg;

struct ClusterTables {
  float2* twM = nullptr;  // per-pass Stockham twiddles of the M-point FFT
  float2* wL = nullptr;   // R x M: w_L^{r k1}
  float2* c = nullptr;    // R x M: e^{-i pi (r + R m)/L}
  float2* wR = nullptr;   // R/2: w_R^{k2}
};

std::mutex g_mu;
std::map<std::pair<int, int>, ClusterTables> g_tabs;  // (device, log2 L)

int ncta_for(int log2L) { return log2L >= 15 ? 16 : 8; }

cudaError_t upload(float2** dst, const std::vector<float2>& v) {
  cudaError_t e = cudaMalloc(dst, sizeof(float2) * v.size());
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), sizeof(float2) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

float2 expi(double ang) { return make_float2(float(std::cos(ang)), float(std::sin(ang))); }

cudaError_t get_cluster_tables(int device, int log2L, ClusterTables* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(device, log2L);
  auto it = g_tabs.find(key);
  if (it != g_tabs.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  const int L = 1 << log2L, R = 2 * ncta_for(log2L), M = L / R;
  std::vector<float2> tw(M, make_float2(0.f, 0.f));
  std::vector<float2> wL(L), c(L), wR(R / 2);
  for (int ns = 8; ns < M; ns *= 8) {  // same per-pass layout as the one-CTA transform
    const int rad = std::min(8, M / ns);
    for (int r = 1; r < rad; ++r)
      for (int k = 0; k < ns; ++k)
        tw[(ns - 8) + (r - 1) * ns + k] = expi(-2.0 * M_PI * double(r) * double(k) / (double(ns) * double(rad)));
  }
  for (int r = 0; r < R; ++r)
    for (int m = 0; m < M; ++m) {
      const long long q = (long long)r * m % L;
      wL[size_t(r) * M + m] = expi(-2.0 * M_PI * double(q) / double(L));
      c[size_t(r) * M + m] = expi(-M_PI * double(r + (long long)R * m) / double(L));
    }
  for (int k = 0; k < R / 2; ++k) wR[k] = expi(-2.0 * M_PI * double(k) / double(R));
  ClusterTables t;
  cudaError_t e = upload(&t.twM, tw);
  if (e == cudaSuccess) e = upload(&t.wL, wL);
  if (e == cudaSuccess) e = upload(&t.c, c);
  if (e == cudaSuccess) e = upload(&t.wR, wR);
  if (e != cudaSuccess) {
    cudaFree(t.twM);
    cudaFree(t.wL);
    cudaFree(t.c);
    cudaFree(t.wR);
    return e;
  }
  g_tabs[key] = t;
  *out = t;
  return cudaSuccess;
}

template <class K>
cudaError_t prepare(K kern, size_t smem, int ncta) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess && ncta > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

void cluster_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, int ncta, int clusters, int threads,
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

template <int LOG2L, int NCTA>
cudaError_t march_t(const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, const ClusterTables& t) {
  using C = CCfg<LOG2L, NCTA>;
  if (cplx) {
    auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, true>;
    cudaError_t e = prepare(k, C::SMEM_CPLX, NCTA);
    if (e != cudaSuccess) return e;
    return launch_cluster(k, NCTA, count, C::NT, C::SMEM_CPLX, st, d, (const float2*)t.twM, (const float2*)t.wL,
                          (const float2*)t.c, (const float2*)t.wR);
  }
  auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, false>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  return launch_cluster(k, NCTA, count, C::NT, C::SMEM, st, d, (const float2*)t.twM, (const float2*)t.wL,
                        (const float2*)t.c, (const float2*)t.wR);
}

template <int LOG2L, int NCTA>
cudaError_t dst_t(const float2* in, float2* out, float scale, int count, long long is, long long os, cudaStream_t st,
                  const ClusterTables& t) {
  using C = CCfg<LOG2L, NCTA>;
  auto k = sssp::sssp_dst_cluster_kernel<LOG2L, NCTA>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  return launch_cluster(k, NCTA, count, C::NT, C::SMEM, st, in, out, scale, (const float2*)t.twM,
                        (const float2*)t.wL, (const float2*)t.c, (const float2*)t.wR, is, os);
}

template <int LOG2L, int NCTA>
cudaError_t fits_t(bool cplx, int* clusters) {
  using C = CCfg<LOG2L, NCTA>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  if (cplx) {
    auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, true>;
    cudaError_t e = prepare(k, C::SMEM_CPLX, NCTA);
    if (e != cudaSuccess) return e;
    cluster_config(&cfg, at, NCTA, 1, C::NT, C::SMEM_CPLX, 0);
    return cudaOccupancyMaxActiveClusters(clusters, k, &cfg);
  }
  auto k = sssp::sssp_march_cluster_kernel<LOG2L, NCTA, false>;
  cudaError_t e = prepare(k, C::SMEM, NCTA);
  if (e != cudaSuccess) return e;
  cluster_config(&cfg, at, NCTA, 1, C::NT, C::SMEM, 0);
  return cudaOccupancyMaxActiveClusters(clusters, k, &cfg);
}

}  // namespace

namespace sssp_cluster {

bool supported(int log2L) { return log2L >= kMinLog2 && log2L <= kMaxLog2; }

int ncta(int log2L) { return ncta_for(log2L); }

cudaError_t max_active_clusters(int log2L, bool cplx, int* clusters) {
  *clusters = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::tuple<int, int, bool>, int> cache;  // (device, log2 L, complex) -> clusters
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, log2L, cplx);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *clusters = it->second;
    return cudaSuccess;
  }
  switch (log2L) {
    case 12: e = fits_t<12, 8>(cplx, clusters); break;
    case 13: e = fits_t<13, 8>(cplx, clusters); break;
    case 14: e = fits_t<14, 8>(cplx, clusters); break;
    case 15: e = fits_t<15, 16>(cplx, clusters); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) cache[key] = *clusters;
  return e;
}

cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, int device) {
  ClusterTables t;
  cudaError_t e = get_cluster_tables(device, log2L, &t);
  if (e != cudaSuccess) return e;
  switch (log2L) {
    case 12: return march_t<12, 8>(d, count, st, cplx, t);
    case 13: return march_t<13, 8>(d, count, st, cplx, t);
    case 14: return march_t<14, 8>(d, count, st, cplx, t);
    case 15: return march_t<15, 16>(d, count, st, cplx, t);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, int count, long long in_stride,
                       long long out_stride, cudaStream_t st, int device) {
  ClusterTables t;
  cudaError_t e = get_cluster_tables(device, log2L, &t);
  if (e != cudaSuccess) return e;
  switch (log2L) {
    case 12: return dst_t<12, 8>(in, out, scale, count, in_stride, out_stride, st, t);
    case 13: return dst_t<13, 8>(in, out, scale, count, in_stride, out_stride, st, t);
    case 14: return dst_t<14, 8>(in, out, scale, count, in_stride, out_stride, st, t);
    case 15: return dst_t<15, 16>(in, out, scale, count, in_stride, out_stride, st, t);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sssp_cluster
