// Host side of the cluster march (march_cluster.cuh): per-shape tables, the default shape of
// every size, the launch with the cluster dimension, and the check that a cluster of a shape
// fits on the device (the other shapes are instantiated in sssp_cluster_shapes.cu).
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

// The default shape of each size: 8 CTAs (16 at L = 32768, whose 8-CTA rows would not fit in
// shared memory); the exchange pushed by remote stores from L = 8192 on and pulled by remote
// loads at L = 4096, the faster of the two at each size as measured (eddy N = 16383: 2.84 s
// pushed against 3.12 s pulled; N = 4095: 312 ms pulled against 320 ms pushed).
int ncta_for(int log2L) { return log2L >= 15 ? 16 : 8; }
bool push_for(int log2L) { return log2L >= 13; }

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

}  // namespace sssp_cluster_host

namespace sssp_cluster {

bool supported(int log2L) { return log2L >= kMinLog2 && log2L <= kMaxLog2; }

int ncta(int log2L) { return ncta_for(log2L); }
bool push_default(int log2L) { return push_for(log2L); }

bool shape_supported(int log2L, int ncta, int push) {
  if (!supported(log2L)) return false;
  if (ncta == 0 || ncta == ncta_for(log2L)) return true;  // the default NCTA, either exchange
  return ncta == 16 && (log2L == 13 || log2L == 14);      // 16-CTA clusters of L = 8192, 16384
}

namespace {
// the explicit shape of a request (0 / -1: the size's default)
void resolve(int log2L, int& ncta, int& push) {
  if (ncta == 0) ncta = ncta_for(log2L);
  if (push < 0) push = push_for(log2L) ? 1 : 0;
}
bool is_default(int log2L, int ncta, int push) { return ncta == ncta_for(log2L) && (push != 0) == push_for(log2L); }
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
  if (!is_default(log2L, ncta, push)) {
    e = sssp_cluster_host::fits_alt(log2L, ncta, push != 0, cplx, clusters);
  } else {
    switch (log2L) {
      case 12: e = fits_t<12, 8, false>(cplx, clusters); break;
      case 13: e = fits_t<13, 8, true>(cplx, clusters); break;
      case 14: e = fits_t<14, 8, true>(cplx, clusters); break;
      case 15: e = fits_t<15, 16, true>(cplx, clusters); break;
      default: return cudaErrorInvalidValue;
    }
  }
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
  if (!is_default(log2L, ncta, push)) return sssp_cluster_host::march_alt(log2L, ncta, push != 0, d, count, st, cplx, t);
  switch (log2L) {
    case 12: return march_t<12, 8, false>(d, count, st, cplx, t);
    case 13: return march_t<13, 8, true>(d, count, st, cplx, t);
    case 14: return march_t<14, 8, true>(d, count, st, cplx, t);
    case 15: return march_t<15, 16, true>(d, count, st, cplx, t);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, int count, long long in_stride,
                       long long out_stride, cudaStream_t st, int device) {
  ClusterTables t;
  cudaError_t e = sssp_cluster_host::get_cluster_tables(device, log2L, ncta_for(log2L), &t);
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
