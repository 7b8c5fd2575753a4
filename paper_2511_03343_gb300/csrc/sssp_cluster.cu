// Host side of the cluster march (march_cluster.cuh): per-shape tables, the default shape of
// every size, the launch with the cluster dimension, the check that a cluster of a shape fits on
// the device, and the 8-CTA shapes (the 16-CTA ones are instantiated in sssp_cluster_shapes.cu).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "cluster_host.cuh"
#include "cluster_launch.h"

namespace {

using sssp_cluster_host::ClusterTables;
using sssp_cluster_host::dst_t;
using sssp_cluster_host::fits_t;
using sssp_cluster_host::march_t;

std::mutex g_mu;
std::map<std::tuple<int, int, int>, ClusterTables> g_tabs;  // (device, log2 L, NCTA)

// The default shape of each size, the fastest of the shapes the autotuner times at every batch
// size measured (1 .. 38 Munk solves, 4 steps), always pulling the exchange: 8 CTAs at L = 4096
// (0.50 ms against 0.51 pushed) and 8192 (0.54 against 0.58 pushed, 0.75 on 16 CTAs); 16 CTAs at
// L = 16384 (alone: 1.02 ms against 1.44 on 8 CTAs pushing; 38 solves: 4.1 against 4.7 ms) and
// 32768 (1.68 against 1.71 pushed; 8-CTA rows would not fit in shared memory there).
int ncta_for(int log2L) { return log2L >= 14 ? 16 : 8; }
bool push_for(int) { return false; }

// CTAs per cluster of the transform-only kernel (pe_dst1 on a cluster plan), a fixed shape:
// 8 CTAs up to L = 16384, 16 at 32768
int dst_ncta(int log2L) { return log2L >= 15 ? 16 : 8; }

cudaError_t upload(float2** dst, const std::vector<float2>& v) {
  cudaError_t e = cudaMalloc(dst, sizeof(float2) * v.size());
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), sizeof(float2) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

float2 expi(double ang) { return make_float2(float(std::cos(ang)), float(std::sin(ang))); }

}  // namespace

namespace sssp_cluster_host {

cudaError_t get_cluster_tables(int device, int log2L, int ncta, ClusterTables* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_tuple(device, log2L, ncta);
  auto it = g_tabs.find(key);
  if (it != g_tabs.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  const int L = 1 << log2L, R = 2 * ncta, M = L / R;
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

cudaError_t march_8(int log2L, bool push, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx,
                    const ClusterTables& t) {
  switch (log2L) {
    case 12: return push ? march_t<12, 8, true>(d, count, st, cplx, t) : march_t<12, 8, false>(d, count, st, cplx, t);
    case 13: return push ? march_t<13, 8, true>(d, count, st, cplx, t) : march_t<13, 8, false>(d, count, st, cplx, t);
    case 14: return push ? march_t<14, 8, true>(d, count, st, cplx, t) : march_t<14, 8, false>(d, count, st, cplx, t);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fits_8(int log2L, bool push, bool cplx, int* clusters) {
  *clusters = 0;
  switch (log2L) {
    case 12: return push ? fits_t<12, 8, true>(cplx, clusters) : fits_t<12, 8, false>(cplx, clusters);
    case 13: return push ? fits_t<13, 8, true>(cplx, clusters) : fits_t<13, 8, false>(cplx, clusters);
    case 14: return push ? fits_t<14, 8, true>(cplx, clusters) : fits_t<14, 8, false>(cplx, clusters);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sssp_cluster_host

namespace sssp_cluster {

bool supported(int log2L) { return log2L >= kMinLog2 && log2L <= kMaxLog2; }

int ncta(int log2L) { return ncta_for(log2L); }
bool push_default(int log2L) { return push_for(log2L); }

bool shape_supported(int log2L, int ncta, int push) {
  if (!supported(log2L) || push < -1 || push > 1) return false;
  if (ncta == 0) return true;                                  // the size's default
  if (ncta == 8) return log2L <= 14;                           // 8-CTA rows fit up to L = 16384
  return ncta == 16 && log2L >= 13;                            // 16-CTA clusters from L = 8192
}

namespace {
// the explicit shape of a request (0 / -1: the size's default)
void resolve(int log2L, int& ncta, int& push) {
  if (ncta == 0) ncta = ncta_for(log2L);
  if (push < 0) push = push_for(log2L) ? 1 : 0;
}
}  // namespace

cudaError_t max_active_clusters(int log2L, bool cplx, int* clusters, int ncta, int push) {
  *clusters = 0;
  if (!shape_supported(log2L, ncta, push)) return cudaErrorInvalidValue;
  resolve(log2L, ncta, push);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  // (device, log2 L, complex, NCTA, push) -> clusters
  static std::map<std::tuple<int, int, bool, int, int>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, log2L, cplx, ncta, push);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *clusters = it->second;
    return cudaSuccess;
  }
  e = ncta == 16 ? sssp_cluster_host::fits_16(log2L, push != 0, cplx, clusters)
                 : sssp_cluster_host::fits_8(log2L, push != 0, cplx, clusters);
  if (e == cudaSuccess) cache[key] = *clusters;
  return e;
}

cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st, bool cplx, int device,
                         int ncta, int push) {
  if (!shape_supported(log2L, ncta, push)) return cudaErrorInvalidValue;
  resolve(log2L, ncta, push);
  ClusterTables t;
  cudaError_t e = sssp_cluster_host::get_cluster_tables(device, log2L, ncta, &t);
  if (e != cudaSuccess) return e;
  return ncta == 16 ? sssp_cluster_host::march_16(log2L, push != 0, d, count, st, cplx, t)
                    : sssp_cluster_host::march_8(log2L, push != 0, d, count, st, cplx, t);
}

cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, int count, long long in_stride,
                       long long out_stride, cudaStream_t st, int device) {
  ClusterTables t;
  cudaError_t e = sssp_cluster_host::get_cluster_tables(device, log2L, dst_ncta(log2L), &t);
  if (e != cudaSuccess) return e;
  switch (log2L) {
    case 12: return dst_t<12, 8, false>(in, out, scale, count, in_stride, out_stride, st, t);
    case 13: return dst_t<13, 8, true>(in, out, scale, count, in_stride, out_stride, st, t);
    case 14: return dst_t<14, 8, true>(in, out, scale, count, in_stride, out_stride, st, t);
    case 15: return dst_t<15, 16, true>(in, out, scale, count, in_stride, out_stride, st, t);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sssp_cluster
