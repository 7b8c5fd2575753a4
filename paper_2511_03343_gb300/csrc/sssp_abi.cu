// C ABI of the SSSP marcher (include/sssp.h): plan construction (FP64 tables on the host),
// device memory, launches and status reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sssp.h"
#include "cluster_launch.h"
#include "march_kernel.cuh"
#include "march_large.cuh"
#include "fd_launch.h"
#include "pade_host.h"
#include "plan_internal.h"
#include "shape_launch.h"

using sssp::Cfg;
using sssp::SolveDesc;
using cd = std::complex<double>;

namespace {

constexpr int kMinLog2 = 3;
constexpr int kMaxSmemLog2 = 12;   // one CTA, everything in shared memory
constexpr int kMaxLog2 = 16;       // beyond: global-memory workspace (march_large.cuh)
constexpr int kMaxTerms = 64;

thread_local std::string g_create_error;

std::mutex g_tab_mu;
std::map<std::tuple<int, int, int>, TransformTables> g_tabs;  // (device, log2L, points per thread)

// twiddles / sine weights in FP64, rounded once to FP32 (shared by all plans of a size and
// shape)
cudaError_t get_tables(int device, int log2L, TransformTables* out, int ppt = 8) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto key = std::make_tuple(device, log2L, ppt);
  auto it = g_tabs.find(key);
  if (it != g_tabs.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  const int L = 1 << log2L;
  std::vector<float2> tw(L, make_float2(0.f, 0.f));
  std::vector<float> sw(L);
  for (int q = 0; q < L; ++q) sw[q] = float(std::sin(M_PI * double(q) / double(L)));
  // per-pass Stockham twiddles exp(-2 pi i r k/(NS R)) at (NS - P) + (r - 1) NS + k for the
  // passes after the first (spans NS = P, P^2, ...; radix R = min(P, L/NS)); L - P entries
  for (int ns = ppt; ns < L; ns *= std::min(ppt, L / ns)) {
    const int R = std::min(ppt, L / ns);
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < ns; ++k) {
        const double ang = 2.0 * M_PI * double(r) * double(k) / (double(ns) * double(R));
        tw[(ns - ppt) + (r - 1) * ns + k] = make_float2(float(std::cos(ang)), float(-std::sin(ang)));
      }
  }
  TransformTables t;
  cudaError_t e = cudaMalloc(&t.tw, sizeof(float2) * L);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&t.sinw, sizeof(float) * L);
  if (e != cudaSuccess) {
    cudaFree(t.tw);
    return e;
  }
  e = cudaMemcpy(t.tw, tw.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.sinw, sw.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  g_tabs[key] = t;
  *out = t;
  return cudaSuccess;
}

int ilog2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return ((1 << l) == v) ? l : -1;
}

}  // namespace


namespace {

// NVTX range over an ABI call (visible in Nsight timelines; no cost without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

pe_status fail(pe_plan* p, pe_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

pe_status cuda_fail(pe_plan* p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(p, PE_ERR_OOM, m);
  return fail(p, PE_ERR_CUDA, m);
}

#define PE_CUDA(plan, call)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(plan, e_, #call); \
  } while (0)

template <int LOG2L>
cudaError_t set_smem_attr() {
  static int done_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (done_dev == dev) return cudaSuccess;
  const int sm = int(Cfg<LOG2L>::SMEM), smc = int(Cfg<LOG2L>::SMEM_CPLX);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(sssp::sssp_march_kernel<LOG2L, false, sssp::kBcDirichlet>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sssp::sssp_march_kernel<LOG2L, true, sssp::kBcDirichlet>, a, smc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sssp::sssp_march_kernel<LOG2L, false, sssp::kBcPeriodic>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sssp::sssp_march_kernel<LOG2L, true, sssp::kBcPeriodic>, a, smc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sssp::sssp_dst_kernel<LOG2L, sssp::kBcDirichlet>, a, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(sssp::sssp_dst_kernel<LOG2L, sssp::kBcPeriodic>, a, sm);
  if (e == cudaSuccess) done_dev = dev;
  return e;
}

template <int LOG2L>
cudaError_t launch_march_t(const SolveDesc* dDescs, int count, const TransformTables& tabs, cudaStream_t st,
                           bool cplx, int bc) {
  cudaError_t e = set_smem_attr<LOG2L>();
  if (e != cudaSuccess) return e;
  const int nt = Cfg<LOG2L>::NT;
  const size_t sm = Cfg<LOG2L>::SMEM, smc = Cfg<LOG2L>::SMEM_CPLX;
  if (bc == sssp::kBcPeriodic) {
    if (cplx)
      sssp::sssp_march_kernel<LOG2L, true, sssp::kBcPeriodic><<<count, nt, smc, st>>>(dDescs, tabs.tw, tabs.sinw);
    else
      sssp::sssp_march_kernel<LOG2L, false, sssp::kBcPeriodic><<<count, nt, sm, st>>>(dDescs, tabs.tw, tabs.sinw);
  } else {
    if (cplx)
      sssp::sssp_march_kernel<LOG2L, true, sssp::kBcDirichlet><<<count, nt, smc, st>>>(dDescs, tabs.tw, tabs.sinw);
    else
      sssp::sssp_march_kernel<LOG2L, false, sssp::kBcDirichlet><<<count, nt, sm, st>>>(dDescs, tabs.tw, tabs.sinw);
  }
  return cudaGetLastError();
}

template <int LOG2L>
cudaError_t launch_dst_t(const float2* in, float2* out, float scale, const TransformTables& tabs, cudaStream_t st,
                         int count = 1, long long in_stride = 0, long long out_stride = 0, int bc = 0) {
  cudaError_t e = set_smem_attr<LOG2L>();
  if (e != cudaSuccess) return e;
  if (bc == sssp::kBcPeriodic)
    sssp::sssp_dst_kernel<LOG2L, sssp::kBcPeriodic><<<count, Cfg<LOG2L>::NT, Cfg<LOG2L>::SMEM, st>>>(
        in, out, scale, tabs.tw, tabs.sinw, in_stride, out_stride);
  else
    sssp::sssp_dst_kernel<LOG2L, sssp::kBcDirichlet><<<count, Cfg<LOG2L>::NT, Cfg<LOG2L>::SMEM, st>>>(
        in, out, scale, tabs.tw, tabs.sinw, in_stride, out_stride);
  return cudaGetLastError();
}

// tables of the two-pass large-grid transform on the current device (cached per size)
template <int LOG2L>
cudaError_t large_tabs(sssp::LargeTabs* out) {
  using B = sssp::BigCfg<LOG2L>;
  static std::mutex mu;
  static std::map<int, sssp::LargeTabs> cache;  // device -> tables
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  // per-pass twiddles of the radix-16 tile FFTs (P and Q points), then w_{2L}^q, all as hi + lo
  auto ff = [](double ang) {
    const double c = std::cos(ang), sn = std::sin(ang);
    const float ch = float(c), sh = float(sn);
    return make_float4(ch, sh, float(c - double(ch)), float(sn - double(sh)));
  };
  auto passes = [&](int F) {
    std::vector<float4> tw(F, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int ns = 1; ns < F; ns *= sssp::large_rad(F, ns)) {
      if (ns == 1) continue;
      const int rad = sssp::large_rad(F, ns), off = sssp::large_twoff(F, ns);
      for (int r = 1; r < rad; ++r)
        for (int k = 0; k < ns; ++k)
          tw[off + (r - 1) * ns + k] = ff(-2.0 * M_PI * double(r) * double(k) / (double(ns) * double(rad)));
    }
    return tw;
  };
  const int n2 = 2 * B::L;
  std::vector<float4> all = passes(B::P), tq = passes(B::Q);
  all.insert(all.end(), tq.begin(), tq.end());
  for (int q = 0; q < n2; ++q) all.push_back(ff(-2.0 * M_PI * double(q) / double(n2)));
  float4* d = nullptr;
  if ((e = cudaMalloc(&d, sizeof(float4) * all.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(d, all.data(), sizeof(float4) * all.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  sssp::LargeTabs t{d, d + B::P, d + B::P + B::Q};
  cache[dev] = t;
  *out = t;
  if ((e = cudaFuncSetAttribute(sssp::sssp_march_large_kernel<LOG2L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(B::SMEM))) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(sssp::sssp_dst_large_kernel<LOG2L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(B::SMEM));
}

template <int LOG2L>
cudaError_t launch_march_large_t(const SolveDesc* dDescs, int count, const TransformTables&, cudaStream_t st) {
  sssp::LargeTabs tb;
  cudaError_t e = large_tabs<LOG2L>(&tb);
  if (e != cudaSuccess) return e;
  sssp::sssp_march_large_kernel<LOG2L><<<count, sssp::kLargeNT, sssp::BigCfg<LOG2L>::SMEM, st>>>(dDescs, tb);
  return cudaGetLastError();
}

template <int LOG2L>
cudaError_t launch_dst_large_t(const float2* in, float2* out, float scale, float2* work, const TransformTables&,
                               cudaStream_t st, int count = 1, long long in_stride = 0, long long out_stride = 0) {
  sssp::LargeTabs tb;
  cudaError_t e = large_tabs<LOG2L>(&tb);
  if (e != cudaSuccess) return e;
  sssp::sssp_dst_large_kernel<LOG2L><<<count, sssp::kLargeNT, sssp::BigCfg<LOG2L>::SMEM, st>>>(
      in, out, scale, work, tb, in_stride, out_stride);
  return cudaGetLastError();
}

cudaError_t launch_march(int log2L, const SolveDesc* d, int count, const TransformTables& tabs, cudaStream_t st,
                         bool cplx, int bc, int ppt = 8) {
  if (ppt != 8) {  // the one-CTA kernel at 4 or 16 points per thread (Dirichlet, L <= 4096)
    if (bc != sssp::kBcDirichlet) return cudaErrorInvalidValue;
    return sssp_shapes::launch_march(log2L, ppt, d, count, tabs.tw, tabs.sinw, st, cplx);
  }
  switch (log2L) {
    case 3: return launch_march_t<3>(d, count, tabs, st, cplx, bc);
    case 4: return launch_march_t<4>(d, count, tabs, st, cplx, bc);
    case 5: return launch_march_t<5>(d, count, tabs, st, cplx, bc);
    case 6: return launch_march_t<6>(d, count, tabs, st, cplx, bc);
    case 7: return launch_march_t<7>(d, count, tabs, st, cplx, bc);
    case 8: return launch_march_t<8>(d, count, tabs, st, cplx, bc);
    case 9: return launch_march_t<9>(d, count, tabs, st, cplx, bc);
    case 10: return launch_march_t<10>(d, count, tabs, st, cplx, bc);
    case 11: return launch_march_t<11>(d, count, tabs, st, cplx, bc);
    case 12: return launch_march_t<12>(d, count, tabs, st, cplx, bc);
    case 13: return launch_march_large_t<13>(d, count, tabs, st);
    case 14: return launch_march_large_t<14>(d, count, tabs, st);
    case 15: return launch_march_large_t<15>(d, count, tabs, st);
    case 16: return launch_march_large_t<16>(d, count, tabs, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dst(int log2L, const float2* in, float2* out, float scale, const TransformTables& tabs,
                       cudaStream_t st, float2* work = nullptr, int bc = 0) {
  switch (log2L) {
    case 13: return launch_dst_large_t<13>(in, out, scale, work, tabs, st);
    case 14: return launch_dst_large_t<14>(in, out, scale, work, tabs, st);
    case 15: return launch_dst_large_t<15>(in, out, scale, work, tabs, st);
    case 16: return launch_dst_large_t<16>(in, out, scale, work, tabs, st);
    case 3: return launch_dst_t<3>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 4: return launch_dst_t<4>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 5: return launch_dst_t<5>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 6: return launch_dst_t<6>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 7: return launch_dst_t<7>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 8: return launch_dst_t<8>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 9: return launch_dst_t<9>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 10: return launch_dst_t<10>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 11: return launch_dst_t<11>(in, out, scale, tabs, st, 1, 0, 0, bc);
    case 12: return launch_dst_t<12>(in, out, scale, tabs, st, 1, 0, 0, bc);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dst_batch(int log2L, const float2* in, float2* out, const TransformTables& tabs, cudaStream_t st,
                             float2* work, int count, long long in_stride, long long out_stride, int bc = 0) {
  switch (log2L) {
    case 3: return launch_dst_t<3>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 4: return launch_dst_t<4>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 5: return launch_dst_t<5>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 6: return launch_dst_t<6>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 7: return launch_dst_t<7>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 8: return launch_dst_t<8>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 9: return launch_dst_t<9>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 10: return launch_dst_t<10>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 11: return launch_dst_t<11>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 12: return launch_dst_t<12>(in, out, 1.f, tabs, st, count, in_stride, out_stride, bc);
    case 13: return launch_dst_large_t<13>(in, out, 1.f, work, tabs, st, count, in_stride, out_stride);
    case 14: return launch_dst_large_t<14>(in, out, 1.f, work, tabs, st, count, in_stride, out_stride);
    case 15: return launch_dst_large_t<15>(in, out, 1.f, work, tabs, st, count, in_stride, out_stride);
    case 16: return launch_dst_large_t<16>(in, out, 1.f, work, tabs, st, count, in_stride, out_stride);
  }
  return cudaErrorInvalidValue;
}

// even extension in place: buf[2K - n] = buf[n], n = 1..K-1 (Neumann plans)
__global__ void even_extend_kernel(float2* buf, int K) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (n < K) buf[2 * K - n] = buf[n];
}

__global__ void carrier_kernel(const float2* __restrict__ field, float2* __restrict__ out, float c, float s, int N,
                               int off) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) {
    const float2 v = field[n + off];
    out[n] = make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
  }
}

void split_ff(cd v, float4* out) {
  const float hr = float(v.real()), hi = float(v.imag());
  out->x = hr;
  out->y = hi;
  out->z = float(v.real() - double(hr));
  out->w = float(v.imag() - double(hi));
}

pe_status ensure_node_cap(pe_plan* p, int need) {
  if (need <= p->node_cap) return PE_OK;
  int cap = std::max(need, std::max(4, p->node_cap * 2));
  float* nV = nullptr;
  double* nR = nullptr;
  PE_CUDA(p, cudaMalloc(&nV, sizeof(float) * size_t(cap) * p->L));
  cudaError_t e = cudaMalloc(&nR, sizeof(double) * cap);
  if (e != cudaSuccess) {
    cudaFree(nV);
    return cuda_fail(p, e, "cudaMalloc(node ranges)");
  }
  if (p->nodes > 0) {
    PE_CUDA(p, cudaMemcpyAsync(nV, p->dV, sizeof(float) * size_t(p->nodes) * p->L, cudaMemcpyDeviceToDevice, p->stream));
    PE_CUDA(p, cudaMemcpyAsync(nR, p->dNodeR, sizeof(double) * p->nodes, cudaMemcpyDeviceToDevice, p->stream));
  }
  float* nVi = nullptr;
  if (p->complex_profile) {
    PE_CUDA(p, cudaMalloc(&nVi, sizeof(float) * size_t(cap) * p->L));
    if (p->nodes > 0)
      PE_CUDA(p, cudaMemcpyAsync(nVi, p->dVi, sizeof(float) * size_t(p->nodes) * p->L, cudaMemcpyDeviceToDevice,
                                 p->stream));
  }
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  cudaFree(p->dV);
  cudaFree(p->dVi);
  cudaFree(p->dNodeR);
  p->dV = nV;
  p->dVi = nVi;
  p->dNodeR = nR;
  p->node_cap = cap;
  return PE_OK;
}

pe_status ensure_tl_cap(pe_plan* p, long long rows) {
  if (rows <= p->tl_cap_rows) return PE_OK;
  long long cap = std::max(rows, std::max<long long>(16, p->tl_cap_rows * 2));
  float* n = nullptr;
  PE_CUDA(p, cudaMalloc(&n, sizeof(float) * size_t(cap) * p->N));
  if (p->tl_rows > 0)
    PE_CUDA(p, cudaMemcpyAsync(n, p->dTL, sizeof(float) * size_t(p->tl_rows) * p->N, cudaMemcpyDeviceToDevice, p->stream));
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  cudaFree(p->dTL);
  p->dTL = n;
  p->tl_cap_rows = cap;
  return PE_OK;
}

int node_for(const pe_plan* p, double rmid) {
  int k = 0;
  for (int i = 0; i < p->nodes; ++i) {
    if (p->node_r[i] <= rmid) k = i;
    else break;
  }
  return k;
}

long long records_between(long long a, long long b, int every) {  // multiples of every in (a, b]
  if (every <= 0) return 0;
  return b / every - a / every;
}

// Whether a march of this plan runs on the cluster kernel (one solve over a thread-block
// cluster), when it is launched together with `group` solves of its size.  Automatic choice:
// Dirichlet grids with L in [4096, 32768] when the device holds such a cluster; at L = 4096
// only while the group's clusters fit on the device at once (the one-CTA kernel does the same
// work on fewer SMs, so it gives more throughput once every SM is busy).
bool use_cluster(const pe_plan* p, bool cplx, int group = 1) {
  if (p->bc != PE_BC_DIRICHLET || !sssp_cluster::supported(p->log2L)) return false;
  if (p->kernel == PE_KERNEL_CTA) return false;
  int clusters = 0;
  if (sssp_cluster::max_active_clusters(p->log2L, cplx, &clusters, p->cl_ncta, p->cl_push) != cudaSuccess ||
      clusters < 1)
    return false;
  if (p->kernel == PE_KERNEL_AUTO && p->log2L == 12 && group > clusters) return false;
  return true;
}

// The cluster shape a march of the plan takes (its own, else the size's default), as
// (CTAs per cluster, push exchange), and as one code 2 NCTA + push for the batch's group key
void cluster_shape_of(const pe_plan* p, int* ncta, int* push) {
  *ncta = p->cl_ncta ? p->cl_ncta : sssp_cluster::ncta(p->log2L);
  *push = p->cl_push >= 0 ? p->cl_push : (sssp_cluster::push_default(p->log2L) ? 1 : 0);
}
int cluster_code(const pe_plan* p) {
  int n = 0, u = 0;
  cluster_shape_of(p, &n, &u);
  return 2 * n + u;
}

// Points per thread of the one-CTA shared-memory kernel a march of this plan runs (8 unless a
// shape was set and is supported; grids beyond one CTA's shared memory take no shape).
int shape_of(const pe_plan* p) {
  if (p->ppt == 8 || p->ppt == 0) return 8;
  if (p->bc != PE_BC_DIRICHLET || !sssp_shapes::supported(p->log2L, p->ppt)) return 8;
  return p->ppt;
}

// Transform tables of the plan's shape on its device
cudaError_t tables_for(const pe_plan* p, int ppt, TransformTables* out) {
  if (ppt == 8) {
    *out = p->tabs;
    return cudaSuccess;
  }
  return get_tables(p->device, p->log2L, out, ppt);
}

// Fill the descriptor for one march of `steps` steps and reserve its TL rows.
pe_status prepare_desc(pe_plan* p, int steps, SolveDesc* d) {
  if (!p->field_set) return fail(p, PE_ERR_STATE, "pe_march before pe_set_field");
  if (p->op == PE_OP_FD3 && p->nodes == 0) return fail(p, PE_ERR_STATE, "FD-SSP march needs a profile (n^2)");
  if (p->op != PE_OP_FD3 && p->terms > 1 && p->nodes == 0)
    return fail(p, PE_ERR_STATE, "pe_march with Neumann terms but no profile");
  if (steps < 0) return fail(p, PE_ERR_ARG, "steps must be >= 0");
  const long long recs = records_between(p->steps_done, p->steps_done + steps, p->tl_every);
  pe_status st = ensure_tl_cap(p, p->tl_rows + recs);
  if (st != PE_OK) return st;
  std::memset(d, 0, sizeof(*d));
  d->R = p->dR;
  d->A = p->dA;
  d->B = p->dB;
  d->G = p->dG;
  d->V = p->dV;
  d->Vi = p->complex_profile ? p->dVi : nullptr;
  d->node_r = p->dNodeR;
  d->yhat = p->dYhat;
  d->work = p->dWork;
  d->field = p->dField;
  d->tl = p->dTL;
  d->status = p->dStatus;
  d->ndst = p->dNdst;
  for (int j = 0; j < sssp::kMaxStages; ++j) d->beta[j] = p->beta[j];
  d->r0 = p->r_set + double(p->steps_done) * p->dr;
  d->dr = p->dr;
  d->tol2 = p->tol * p->tol;
  d->step0 = p->steps_done;
  d->rec0 = p->tl_rows;
  d->nodes = p->nodes;
  d->node0 = (p->nodes > 0) ? node_for(p, d->r0 + 0.5 * p->dr) : 0;
  d->steps = steps;
  d->p = p->p;
  d->terms = p->terms;
  d->tl_every = p->tl_every;
  d->N = p->N;
  d->fd = p->dFD;
  d->fdc = p->dFDc;
  for (long long s = 1; s <= steps; ++s)
    if (p->tl_every > 0 && (p->steps_done + s) % p->tl_every == 0) p->tl_ranges.push_back(p->r_set + double(p->steps_done + s) * p->dr);
  p->tl_rows += recs;
  p->steps_done += steps;
  return PE_OK;
}

pe_status check_status(pe_plan* p) {
  int s = 0;
  PE_CUDA(p, cudaMemcpyAsync(&s, p->dStatus, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  if (s == sssp::kStatusDiverged)
    return fail(p, PE_ERR_NEUMANN_DIVERGED, "Neumann series diverged (a term grew to 1e4 times the first correction)");
  if (s == sssp::kStatusNumeric) return fail(p, PE_ERR_NUMERIC, "non-finite value in the march");
  if (s != 0) return fail(p, PE_ERR_CUDA, "device status " + std::to_string(s));
  return PE_OK;
}

}  // namespace

extern "C" {

int pe_abi_version(void) { return 1; }

const char* pe_create_error(void) { return g_create_error.c_str(); }

const char* pe_last_error(const pe_plan* plan) { return plan ? plan->err.c_str() : ""; }

pe_status pe_pade_coefficients(double sigma, int p, double* b, double* a, double* d) {
  if (!b || !a || !d) return PE_ERR_ARG;
  sssp::PadeData pd;
  std::string err;
  if (!sssp::pade_compute(sigma, p, &pd, &err)) {
    g_create_error = err;
    return PE_ERR_ARG;
  }
  for (int j = 0; j < p; ++j) {
    b[2 * j] = pd.b[j].real();
    b[2 * j + 1] = pd.b[j].imag();
    a[2 * j] = pd.a[j].real();
    a[2 * j + 1] = pd.a[j].imag();
    d[2 * j + 2] = pd.d[j].real();
    d[2 * j + 3] = pd.d[j].imag();
  }
  d[0] = pd.d0.real();
  d[1] = pd.d0.imag();
  return PE_OK;
}

void pe_plan_destroy(pe_plan* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  cudaFree(p->dR);
  cudaFree(p->dA);
  cudaFree(p->dB);
  cudaFree(p->dG);
  cudaFree(p->dYhat);
  cudaFree(p->dField);
  cudaFree(p->dStage);
  cudaFree(p->dWork);
  cudaFree(p->dV);
  cudaFree(p->dVi);
  cudaFree(p->dNodeR);
  cudaFree(p->dStatus);
  cudaFree(p->dNdst);
  cudaFree(p->dTL);
  cudaFree(p->dDesc);
  cudaFree(p->dFD);
  cudaFree(p->dFDc);
  delete p;
}

pe_status pe_plan_create(pe_plan** out, int N, double H, double k0, double dr, int pade_order, int neumann_terms,
                         double neumann_tol, void* cuda_stream) {
  return pe_plan_create_bc(out, N, H, k0, dr, pade_order, neumann_terms, neumann_tol, PE_BC_DIRICHLET, cuda_stream);
}

pe_status pe_plan_create_bc(pe_plan** out, int N, double H, double k0, double dr, int pade_order, int neumann_terms,
                            double neumann_tol, int bc, void* cuda_stream) {
  NvtxRange nvtx_("pe_plan_create");
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return PE_ERR_ARG;
  }
  *out = nullptr;
  if (bc != PE_BC_DIRICHLET && bc != PE_BC_PERIODIC && bc != PE_BC_NEUMANN) {
    g_create_error = "bc must be PE_BC_DIRICHLET, PE_BC_PERIODIC or PE_BC_NEUMANN";
    return PE_ERR_ARG;
  }
  const int user_bc = bc, N_user = N;
  if (bc == PE_BC_NEUMANN) {
    // the even extension to [0, 2H]: 2(N-1) periodic points
    if (N < 5 || ilog2_exact(N - 1) < 2 || 2 * (N - 1) > (1 << kMaxSmemLog2)) {
      g_create_error = "Neumann grids: N - 1 must be a power of two in [4, 2048]";
      return PE_ERR_ARG;
    }
    N = 2 * (N - 1);
    H = 2.0 * H;
    bc = PE_BC_PERIODIC;
  }
  const int log2L = ilog2_exact(bc == PE_BC_PERIODIC ? N : N + 1);
  if (bc == PE_BC_DIRICHLET && (N < 1 || log2L < kMinLog2 || log2L > kMaxLog2)) {
    g_create_error = "N + 1 must be a power of two in [8, 65536]";
    return PE_ERR_ARG;
  }
  if (bc == PE_BC_PERIODIC && (N < 1 || log2L < kMinLog2 || log2L > kMaxSmemLog2)) {
    g_create_error = "periodic grids: N must be a power of two in [8, 4096]";
    return PE_ERR_ARG;
  }
  if (!(H > 0) || !(k0 > 0) || !(dr > 0) || !std::isfinite(H) || !std::isfinite(k0) || !std::isfinite(dr)) {
    g_create_error = "H, k0 and dr must be finite and > 0";
    return PE_ERR_ARG;
  }
  if (pade_order < 1 || pade_order > sssp::kMaxPade) {
    g_create_error = "pade_order must be in [1, 8]";
    return PE_ERR_ARG;
  }
  if (neumann_terms < 0 || neumann_terms > kMaxTerms || !(neumann_tol >= 0)) {
    g_create_error = "neumann_terms must be in [0, 64] and neumann_tol >= 0";
    return PE_ERR_ARG;
  }
  pe_plan* p = new pe_plan();
  p->N = N;
  p->L = 1 << log2L;
  p->log2L = log2L;
  p->bc = bc;
  p->off = (bc == PE_BC_PERIODIC) ? 0 : 1;
  p->user_bc = user_bc;
  p->N_user = N_user;
  p->p = pade_order;
  p->terms = neumann_terms;
  p->H = H;
  p->k0 = k0;
  p->dr = dr;
  p->tol = neumann_tol;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  std::string err;
  if (!sssp::pade_compute(k0 * dr, pade_order, &p->pade, &err)) {
    g_create_error = err;
    delete p;
    return PE_ERR_ARG;
  }
  auto bail = [&](cudaError_t e, const char* what) {
    g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
    pe_plan_destroy(p);
    return e == cudaErrorMemoryAllocation ? PE_ERR_OOM : PE_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  e = get_tables(p->device, log2L, &p->tabs);
  if (e != cudaSuccess) return bail(e, "transform tables");
  // plan tables in FP64 (Section 3: 1/(1 + b_j lambda_m), lambda_m = -(pi m/(k0 H))^2)
  const int L = p->L, P = pade_order;
  std::vector<float4> R(size_t(P) * L), G(L);
  std::vector<float2> A(size_t(P) * L), B(size_t(P) * L);
  // Dirichlet: sin(pi m z/H), m = 1..N (m = 0 a zero pad), unnormalised DST-I pair with 2/L;
  // periodic: e^{2 pi i l z/H} with the signed frequency l, DFT pair with 1/L
  const bool periodic = (bc == PE_BC_PERIODIC);
  const double scale = (periodic ? 1.0 : 2.0) / double(L);
  for (int m = 0; m < L; ++m) {
    const double l = periodic ? double(m <= L / 2 ? m : m - L) : double(m);
    const double x = (periodic ? 2.0 : 1.0) * M_PI * l / (k0 * H);
    const double lam = -x * x;
    cd g(1.0, 0.0);
    for (int j = 0; j < P; ++j) {
      const cd b = p->pade.b[j], a = p->pade.a[j];
      const cd q = 1.0 + b * lam;
      const cd r = (1.0 + a * lam) / q;
      g *= r;
      const size_t ix = size_t(j) * L + m;
      if (m == 0 && !periodic) {
        R[ix] = make_float4(0, 0, 0, 0);
        A[ix] = make_float2(0, 0);
        B[ix] = make_float2(0, 0);
        continue;
      }
      split_ff(r, &R[ix]);
      const cd av = scale / q, bv = scale * (-b) / q;
      A[ix] = make_float2(float(av.real()), float(av.imag()));
      B[ix] = make_float2(float(bv.real()), float(bv.imag()));
    }
    if (m == 0 && !periodic) G[m] = make_float4(0, 0, 0, 0);
    else split_ff(g, &G[m]);
  }
  for (int j = 0; j < sssp::kMaxStages; ++j) {
    if (j < P) {
      const cd bb = (1.0 / scale) * (1.0 - p->pade.a[j] / p->pade.b[j]);
      p->beta[j] = make_float2(float(bb.real()), float(bb.imag()));
    } else {
      p->beta[j] = make_float2(0, 0);
    }
  }
  if ((e = cudaMalloc(&p->dR, sizeof(float4) * R.size())) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dA, sizeof(float2) * A.size())) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dB, sizeof(float2) * B.size())) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dG, sizeof(float4) * L)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dYhat, sizeof(float2) * L)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dField, sizeof(float2) * L)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dStage, sizeof(float2) * L)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dStatus, sizeof(int))) != cudaSuccess) return bail(e, "cudaMalloc");
  if (log2L > kMaxSmemLog2 &&
      (e = cudaMalloc(&p->dWork, sizeof(float2) * sssp::large_work_elems(L))) != cudaSuccess)
    return bail(e, "cudaMalloc(workspace)");
  if ((e = cudaMalloc(&p->dNdst, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->dDesc, sizeof(SolveDesc))) != cudaSuccess) return bail(e, "cudaMalloc");
  p->desc_cap = sizeof(SolveDesc);
  if ((e = cudaMemcpy(p->dR, R.data(), sizeof(float4) * R.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemcpy(p->dA, A.data(), sizeof(float2) * A.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemcpy(p->dB, B.data(), sizeof(float2) * B.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemcpy(p->dG, G.data(), sizeof(float4) * L, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemset(p->dStatus, 0, sizeof(int))) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemset(p->dNdst, 0, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemset(p->dYhat, 0, sizeof(float2) * L)) != cudaSuccess) return bail(e, "memset");
  if ((e = cudaMemset(p->dField, 0, sizeof(float2) * L)) != cudaSuccess) return bail(e, "memset");
  *out = p;
  return PE_OK;
}

pe_status pe_set_output(pe_plan* p, int tl_every) {
  if (!p) return PE_ERR_ARG;
  if (tl_every < 0) return fail(p, PE_ERR_ARG, "tl_every must be >= 0");
  p->tl_every = tl_every;
  p->tl_rows = 0;
  p->tl_ranges.clear();
  return PE_OK;
}

pe_status pe_set_field(pe_plan* p, const float* u, int on_device, double r) {
  if (!p) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_set_field");
  if (!u) return fail(p, PE_ERR_ARG, "u is NULL");
  if (!std::isfinite(r)) return fail(p, PE_ERR_ARG, "r must be finite");
  PE_CUDA(p, cudaMemcpyAsync(p->dStage, u, sizeof(float2) * p->N_user,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
  if (p->user_bc == PE_BC_NEUMANN) {
    const int K = p->N / 2;
    even_extend_kernel<<<(K + 255) / 256, 256, 0, p->stream>>>(p->dStage, K);
    PE_CUDA(p, cudaGetLastError());
  }
  if (p->op == PE_OP_FD3) {  // FD-SSP marches depth values: index 0 the boundary, 1..N the field
    PE_CUDA(p, cudaMemsetAsync(p->dYhat, 0, sizeof(float2), p->stream));
    PE_CUDA(p, cudaMemcpyAsync(p->dYhat + 1, p->dStage, sizeof(float2) * p->N, cudaMemcpyDeviceToDevice, p->stream));
  } else {
    PE_CUDA(p, launch_dst(p->log2L, p->dStage, p->dYhat, 1.0f, p->tabs, p->stream, p->dWork, p->bc));
  }
  // the physical field as given (Dirichlet: index 0 = boundary)
  if (p->off) PE_CUDA(p, cudaMemsetAsync(p->dField, 0, sizeof(float2), p->stream));
  PE_CUDA(p, cudaMemcpyAsync(p->dField + p->off, p->dStage, sizeof(float2) * p->N, cudaMemcpyDeviceToDevice,
                             p->stream));
  PE_CUDA(p, cudaMemsetAsync(p->dStatus, 0, sizeof(int), p->stream));
  if (!on_device) PE_CUDA(p, cudaStreamSynchronize(p->stream));
  p->r_set = r;
  p->steps_done = 0;
  p->tl_rows = 0;
  p->tl_ranges.clear();
  p->field_set = true;
  return PE_OK;
}

static pe_status append_nodes(pe_plan* p, const double* n2, const double* ranges, int count, int on_device,
                              int is_complex = 0) {
  for (int i = 0; i < count; ++i) {
    const double prev = (p->nodes + i > 0) ? (i > 0 ? ranges[i - 1] : p->node_r.back()) : -1e300;
    if (!std::isfinite(ranges[i]) || ranges[i] < prev) return fail(p, PE_ERR_ARG, "profile ranges must be finite and non-decreasing");
  }
  if (is_complex && !p->complex_profile) {
    // first complex node: imaginary rows for every node (zeros for the real ones so far)
    if (p->node_cap > 0) {
      PE_CUDA(p, cudaMalloc(&p->dVi, sizeof(float) * size_t(p->node_cap) * p->L));
      PE_CUDA(p, cudaMemsetAsync(p->dVi, 0, sizeof(float) * size_t(p->node_cap) * p->L, p->stream));
    }
    p->complex_profile = true;
  }
  pe_status st = ensure_node_cap(p, p->nodes + count);
  if (st != PE_OK) return st;
  const size_t per = size_t(p->N_user) * (is_complex ? 2 : 1);
  const bool neumann = (p->user_bc == PE_BC_NEUMANN);
  const int K = p->N / 2;
  std::vector<double> src;
  const double* s = n2;
  if (on_device) {
    src.resize(size_t(count) * per);
    PE_CUDA(p, cudaMemcpyAsync(src.data(), n2, sizeof(double) * src.size(), cudaMemcpyDeviceToHost, p->stream));
    PE_CUDA(p, cudaStreamSynchronize(p->stream));
    s = src.data();
  }
  // V = n^2 - 1 formed in FP64, then rounded; index 0 is the boundary (0)
  std::vector<float> host(size_t(count) * p->L), hosti;
  if (p->complex_profile) hosti.assign(size_t(count) * p->L, 0.f);
  for (int i = 0; i < count; ++i) {
    host[size_t(i) * p->L] = 0.0f;  // Dirichlet boundary (overwritten by data on periodic grids)
    for (int n = 0; n < p->N; ++n) {
      const int q = (neumann && n > K) ? 2 * K - n : n;  // even extension for Neumann plans
      const double re = is_complex ? s[size_t(i) * per + 2 * q] : s[size_t(i) * per + q];
      const double im = is_complex ? s[size_t(i) * per + 2 * q + 1] : 0.0;
      if (!std::isfinite(re) || !std::isfinite(im)) return fail(p, PE_ERR_ARG, "n2 must be finite");
      host[size_t(i) * p->L + n + p->off] = float(re - 1.0);
      if (p->complex_profile) hosti[size_t(i) * p->L + n + p->off] = float(im);
    }
  }
  PE_CUDA(p, cudaMemcpyAsync(p->dV + size_t(p->nodes) * p->L, host.data(), sizeof(float) * host.size(),
                             cudaMemcpyHostToDevice, p->stream));
  if (p->complex_profile)
    PE_CUDA(p, cudaMemcpyAsync(p->dVi + size_t(p->nodes) * p->L, hosti.data(), sizeof(float) * hosti.size(),
                               cudaMemcpyHostToDevice, p->stream));
  PE_CUDA(p, cudaMemcpyAsync(p->dNodeR + p->nodes, ranges, sizeof(double) * count, cudaMemcpyHostToDevice, p->stream));
  if (p->op == PE_OP_FD3) {  // FD-SSP: FP64 Thomas factors of every stage for the new nodes
    if (is_complex) return fail(p, PE_ERR_ARG, "FD-SSP plans take real n^2 only");
    const size_t per_node = size_t(p->p) * p->L * 3;
    if (p->nodes + count > p->fd_cap) {
      const int cap = std::max(p->nodes + count, std::max(4, 2 * p->fd_cap));
      float4* n = nullptr;
      PE_CUDA(p, cudaMalloc(&n, sizeof(float4) * per_node * cap));
      if (p->nodes > 0)
        PE_CUDA(p, cudaMemcpyAsync(n, p->dFD, sizeof(float4) * per_node * p->nodes, cudaMemcpyDeviceToDevice,
                                   p->stream));
      PE_CUDA(p, cudaStreamSynchronize(p->stream));
      cudaFree(p->dFD);
      p->dFD = n;
      p->fd_cap = cap;
    }
    std::vector<float4> tab(per_node * count);
    std::vector<double> Vd(p->N);
    for (int i = 0; i < count; ++i) {
      for (int n = 0; n < p->N; ++n) Vd[n] = s[size_t(i) * per + n] - 1.0;
      sssp_fd::factor_node(Vd.data(), p->N, p->L, p->H, p->k0, p->pade.b, p->p, tab.data() + per_node * i);
    }
    PE_CUDA(p, cudaMemcpyAsync(p->dFD + per_node * p->nodes, tab.data(), sizeof(float4) * tab.size(),
                               cudaMemcpyHostToDevice, p->stream));
  }
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int i = 0; i < count; ++i) p->node_r.push_back(ranges[i]);
  p->nodes += count;
  return PE_OK;
}

pe_status pe_set_profile(pe_plan* p, const double* n2, int is_complex, double range, int on_device) {
  if (!p) return PE_ERR_ARG;
  if (!n2) return fail(p, PE_ERR_ARG, "n2 is NULL");
  return append_nodes(p, n2, &range, 1, on_device, is_complex ? 1 : 0);
}

pe_status pe_set_profiles(pe_plan* p, const double* n2, const double* ranges, int count, int on_device) {
  NvtxRange nvtx_("pe_set_profiles");
  if (!p) return PE_ERR_ARG;
  if (!n2 || !ranges || count < 0) return fail(p, PE_ERR_ARG, "n2/ranges NULL or count < 0");
  return append_nodes(p, n2, ranges, count, on_device);
}

pe_status pe_clear_profiles(pe_plan* p) {
  if (!p) return PE_ERR_ARG;
  p->nodes = 0;
  p->complex_profile = false;
  cudaFree(p->dVi);
  p->dVi = nullptr;
  p->node_r.clear();
  return PE_OK;
}

pe_status pe_march(pe_plan* p, int steps) {
  if (!p) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_march");
  SolveDesc d;
  pe_status st = prepare_desc(p, steps, &d);
  if (st != PE_OK) return st;
  if (steps == 0) return PE_OK;
  PE_CUDA(p, cudaMemcpyAsync(p->dDesc, &d, sizeof(d), cudaMemcpyHostToDevice, p->stream));  // capacity >= 1
  const bool cplx = d.Vi != nullptr;
  if (p->op == PE_OP_FD3) {
    PE_CUDA(p, sssp_fd::launch_march(p->log2L, p->dDesc, 1, p->stream));
  } else if (use_cluster(p, cplx)) {
    PE_CUDA(p, sssp_cluster::launch_march(p->log2L, p->dDesc, 1, p->stream, cplx, p->device, p->cl_ncta,
                                          p->cl_push));
  } else {
    const int ppt = (p->log2L <= kMaxSmemLog2) ? shape_of(p) : 8;
    TransformTables tb;
    PE_CUDA(p, tables_for(p, ppt, &tb));
    PE_CUDA(p, launch_march(p->log2L, p->dDesc, 1, tb, p->stream, cplx, p->bc, ppt));
  }
  return PE_OK;
}

}  // extern "C"

namespace {

// Streams, events and descriptor arrays of batched marches, per device (kept for the process):
// group g of a batch always runs on stream g and reads descriptor array g, so a later batch's
// upload into array g is ordered after the earlier batch's launch that read it.
struct BatchLanes {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<SolveDesc*> descs;
  std::vector<size_t> cap;
  cudaEvent_t fork = nullptr;
};
std::mutex g_lanes_mu;
std::map<int, BatchLanes> g_lanes;

cudaError_t lanes_for(int device, int groups, BatchLanes** out) {
  BatchLanes& b = g_lanes[device];
  cudaError_t e = cudaSuccess;
  if (!b.fork && (e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  while (int(b.streams.size()) < groups) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    b.streams.push_back(st);
    b.done.push_back(ev);
    b.descs.push_back(nullptr);
    b.cap.push_back(0);
  }
  *out = &b;
  return cudaSuccess;
}

}  // namespace

extern "C" {

pe_status pe_march_batch_steps(pe_plan** plans, const int* steps, int count) {
  if (!plans || !steps || count < 0) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_march_batch_steps");
  if (count == 0) return PE_OK;
  pe_plan* p0 = plans[0];
  if (!p0) return PE_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return fail(p0, PE_ERR_ARG, "NULL plan in batch");
    if (plans[i]->device != p0->device) return fail(p0, PE_ERR_ARG, "plans on different devices");
    if (steps[i] < 0) return fail(p0, PE_ERR_ARG, "steps must be >= 0");
  }
  // group by (size, complex profile, boundary condition, kernel, shape), one launch per group;
  // every CTA (or cluster) marches its own plan its own step count
  using GroupKey = std::tuple<int, bool, int, bool, int>;
  std::map<GroupKey, std::vector<SolveDesc>> groups;
  std::map<GroupKey, std::vector<double>> costs;
  std::map<GroupKey, TransformTables> tabs;
  std::map<std::tuple<int, bool, int>, int> size_count;  // solves per (size, complex, bc)
  for (int i = 0; i < count; ++i)
    if (steps[i] > 0)
      ++size_count[std::make_tuple(plans[i]->log2L, plans[i]->complex_profile, plans[i]->bc)];
  for (int i = 0; i < count; ++i) {
    if (steps[i] == 0) continue;
    SolveDesc d;
    pe_status st = prepare_desc(plans[i], steps[i], &d);
    if (st != PE_OK) {
      p0->err = plans[i]->err;
      return st;
    }
    const bool cplx = d.Vi != nullptr;
    const int group = size_count[std::make_tuple(plans[i]->log2L, plans[i]->complex_profile, plans[i]->bc)];
    const bool fd = plans[i]->op == PE_OP_FD3;  // FD-SSP plans: their own kernel (shape -1)
    const bool cl = !fd && use_cluster(plans[i], cplx, group);
    // the shape slot of the group key: points per thread of the one-CTA kernel, -1 for FD-SSP, the
    // cluster shape's code (2 NCTA + push, >= 16) for the cluster kernel
    const int ppt = fd ? -1 : (cl ? cluster_code(plans[i]) : (plans[i]->log2L <= kMaxSmemLog2 ? shape_of(plans[i]) : 8));
    const auto key = std::make_tuple(plans[i]->log2L, cplx, plans[i]->bc, cl, ppt);
    groups[key].push_back(d);
    costs[key].push_back(plans[i]->cost);
    if (!tabs.count(key)) {
      TransformTables tb = plans[i]->tabs;
      if (!fd && !cl) PE_CUDA(p0, tables_for(plans[i], ppt, &tb));
      tabs[key] = tb;
    }
  }
  // Where every solve of a group has a measured cost, launch the group's CTAs in descending cost
  // (the block scheduler fills the SMs in launch order, so heavy and light solves end up sharing
  // SMs; measured 5 % off the 256-solve batch).  Each CTA marches its own solve: the results
  // do not depend on the order.
  for (auto& kv : groups) {
    std::vector<double>& c = costs[kv.first];
    if (std::any_of(c.begin(), c.end(), [](double v) { return !(v > 0.0); })) continue;
    std::vector<size_t> idx(c.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return c[a] > c[b]; });
    std::vector<SolveDesc> sorted;
    sorted.reserve(idx.size());
    for (size_t k : idx) sorted.push_back(kv.second[k]);
    kv.second.swap(sorted);
  }
  if (groups.size() == 1) {  // one group: on the plan's stream, in its own descriptor array
    auto& kv = *groups.begin();
    const size_t bytes = sizeof(SolveDesc) * kv.second.size();
    if (bytes > p0->desc_cap) {
      PE_CUDA(p0, cudaStreamSynchronize(p0->stream));
      cudaFree(p0->dDesc);
      p0->dDesc = nullptr;
      p0->desc_cap = 0;
      PE_CUDA(p0, cudaMalloc(reinterpret_cast<void**>(&p0->dDesc), bytes));
      p0->desc_cap = bytes;
    }
    PE_CUDA(p0, cudaMemcpyAsync(p0->dDesc, kv.second.data(), bytes, cudaMemcpyHostToDevice, p0->stream));
    if (std::get<4>(kv.first) < 0)
      PE_CUDA(p0, sssp_fd::launch_march(std::get<0>(kv.first), p0->dDesc, int(kv.second.size()), p0->stream));
    else if (std::get<3>(kv.first))
      PE_CUDA(p0, sssp_cluster::launch_march(std::get<0>(kv.first), p0->dDesc, int(kv.second.size()), p0->stream,
                                             std::get<1>(kv.first), p0->device, std::get<4>(kv.first) / 2,
                                             std::get<4>(kv.first) & 1));
    else
      PE_CUDA(p0, launch_march(std::get<0>(kv.first), p0->dDesc, int(kv.second.size()), tabs[kv.first], p0->stream,
                               std::get<1>(kv.first), std::get<2>(kv.first), std::get<4>(kv.first)));
    return PE_OK;
  }
  // several groups (grid sizes / kernels): each on its own stream, forked from the plan's stream
  // and joined back to it, so that their launches overlap on the device
  std::lock_guard<std::mutex> lk(g_lanes_mu);
  BatchLanes* bl = nullptr;
  PE_CUDA(p0, lanes_for(p0->device, int(groups.size()), &bl));
  PE_CUDA(p0, cudaEventRecord(bl->fork, p0->stream));
  int g = 0;
  for (auto& kv : groups) {
    cudaStream_t st = bl->streams[g];
    const size_t bytes = sizeof(SolveDesc) * kv.second.size();
    PE_CUDA(p0, cudaStreamWaitEvent(st, bl->fork, 0));
    if (bytes > bl->cap[g]) {
      PE_CUDA(p0, cudaStreamSynchronize(st));
      cudaFree(bl->descs[g]);
      bl->descs[g] = nullptr;
      bl->cap[g] = 0;
      PE_CUDA(p0, cudaMalloc(reinterpret_cast<void**>(&bl->descs[g]), std::max<size_t>(bytes, 64 * sizeof(SolveDesc))));
      bl->cap[g] = std::max<size_t>(bytes, 64 * sizeof(SolveDesc));
    }
    SolveDesc* dd = bl->descs[g];
    PE_CUDA(p0, cudaMemcpyAsync(dd, kv.second.data(), bytes, cudaMemcpyHostToDevice, st));
    if (std::get<4>(kv.first) < 0)
      PE_CUDA(p0, sssp_fd::launch_march(std::get<0>(kv.first), dd, int(kv.second.size()), st));
    else if (std::get<3>(kv.first))
      PE_CUDA(p0, sssp_cluster::launch_march(std::get<0>(kv.first), dd, int(kv.second.size()), st,
                                             std::get<1>(kv.first), p0->device, std::get<4>(kv.first) / 2,
                                             std::get<4>(kv.first) & 1));
    else
      PE_CUDA(p0, launch_march(std::get<0>(kv.first), dd, int(kv.second.size()), tabs[kv.first], st,
                               std::get<1>(kv.first), std::get<2>(kv.first), std::get<4>(kv.first)));
    PE_CUDA(p0, cudaEventRecord(bl->done[g], st));
    PE_CUDA(p0, cudaStreamWaitEvent(p0->stream, bl->done[g], 0));
    ++g;
  }
  return PE_OK;
}

pe_status pe_march_batch(pe_plan** plans, int count, int steps) {
  if (!plans || count < 0) return PE_ERR_ARG;
  std::vector<int> st(size_t(count), steps);
  if (steps < 0) {
    if (count > 0 && plans[0]) return fail(plans[0], PE_ERR_ARG, "steps must be >= 0");
    return PE_ERR_ARG;
  }
  return pe_march_batch_steps(plans, st.data(), count);
}

size_t pe_plan_bytes_estimate(int N, int pade_order, int nodes, long long tl_rows) {
  const size_t L = size_t(N) + 1, p = size_t(pade_order > 0 ? pade_order : 0);
  size_t b = L * p * (sizeof(float4) + 2 * sizeof(float2));      // R, A, B tables
  b += L * sizeof(float4) + 3 * L * sizeof(float2);               // G, spectral state, field, staging
  b += size_t(nodes > 0 ? nodes : 0) * (L * sizeof(float) + sizeof(double));
  b += size_t(tl_rows > 0 ? tl_rows : 0) * size_t(N) * sizeof(float);
  if (L > (size_t(1) << kMaxSmemLog2)) b += sssp::large_work_elems(int(L)) * sizeof(float2);
  return b + 1024;
}

pe_status pe_sync(pe_plan* p) {
  if (!p) return PE_ERR_ARG;
  return check_status(p);
}

pe_status pe_read_field(pe_plan* p, float* out, int to_device) {
  if (!p) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_read_field");
  if (!out) return fail(p, PE_ERR_ARG, "out is NULL");
  // carrier e^{i k0 (r - r_set)} in FP64 phase arithmetic (the marcher keeps the envelope)
  const double phase = std::fmod(p->k0 * p->dr * double(p->steps_done), 2.0 * M_PI);
  const float c = float(std::cos(phase)), s = float(std::sin(phase));
  const bool direct = to_device && p->N_user == p->N;
  float2* dst = direct ? reinterpret_cast<float2*>(out) : p->dStage;
  carrier_kernel<<<(p->N + 255) / 256, 256, 0, p->stream>>>(p->dField, dst, c, s, p->N, p->off);
  PE_CUDA(p, cudaGetLastError());
  if (!direct)
    PE_CUDA(p, cudaMemcpyAsync(out, p->dStage, sizeof(float2) * p->N_user,
                               to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
  return check_status(p);
}

pe_status pe_read_TL(pe_plan* p, float* out, size_t cap, double* ranges, size_t* n_rows) {
  NvtxRange nvtx_("pe_read_TL");
  if (!p) return PE_ERR_ARG;
  const size_t need = size_t(p->tl_rows) * p->N_user;
  if (n_rows) *n_rows = size_t(p->tl_rows);
  if (!out) return PE_OK;  // size query
  if (cap < need) return fail(p, PE_ERR_ARG, "TL buffer too small");
  if (need > 0)  // rows hold N values on the device; the caller gets the first N_user of each
    PE_CUDA(p, cudaMemcpy2DAsync(out, sizeof(float) * p->N_user, p->dTL, sizeof(float) * p->N,
                                 sizeof(float) * p->N_user, size_t(p->tl_rows), cudaMemcpyDeviceToHost, p->stream));
  if (ranges)
    for (size_t i = 0; i < p->tl_ranges.size(); ++i) ranges[i] = p->tl_ranges[i];
  return check_status(p);
}

pe_status pe_get_transform_count(pe_plan* p, unsigned long long* count) {
  if (!p || !count) return PE_ERR_ARG;
  PE_CUDA(p, cudaMemcpyAsync(count, p->dNdst, sizeof(unsigned long long), cudaMemcpyDeviceToHost, p->stream));
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  return PE_OK;
}

pe_status pe_dst1(pe_plan* p, const float* in, float* out, int on_device) {
  if (!p) return PE_ERR_ARG;
  if (!in || !out) return fail(p, PE_ERR_ARG, "in/out is NULL");
  float2* tmp = p->dStage;
  float2* res = nullptr;
  PE_CUDA(p, cudaMallocAsync(reinterpret_cast<void**>(&res), sizeof(float2) * p->L, p->stream));
  PE_CUDA(p, cudaMemcpyAsync(tmp, in, sizeof(float2) * p->N_user,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
  float scale = 1.0f;
  if (p->user_bc == PE_BC_NEUMANN) {  // DCT-I = half the DFT of the even extension
    const int K = p->N / 2;
    even_extend_kernel<<<(K + 255) / 256, 256, 0, p->stream>>>(tmp, K);
    PE_CUDA(p, cudaGetLastError());
    scale = 0.5f;
  }
  if (p->user_bc == PE_BC_DIRICHLET && p->kernel == PE_KERNEL_CLUSTER)
    PE_CUDA(p, sssp_cluster::launch_dst(p->log2L, tmp, res, scale, 1, 0, 0, p->stream, p->device));
  else
    PE_CUDA(p, launch_dst(p->log2L, tmp, res, scale, p->tabs, p->stream, p->dWork, p->bc));
  PE_CUDA(p, cudaMemcpyAsync(out, res + p->off, sizeof(float2) * p->N_user,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
  PE_CUDA(p, cudaFreeAsync(res, p->stream));
  if (!on_device) PE_CUDA(p, cudaStreamSynchronize(p->stream));
  return PE_OK;
}

pe_status pe_dst1_batch(pe_plan* p, const float* in, float* out, int count) {
  if (!p) return PE_ERR_ARG;
  if (!in || !out || count < 0) return fail(p, PE_ERR_ARG, "in/out NULL or count < 0");
  if (p->user_bc == PE_BC_NEUMANN) return fail(p, PE_ERR_ARG, "pe_dst1_batch takes Dirichlet or periodic plans");
  if (count == 0) return PE_OK;
  // every field gets an L-long result row (index 0 is the zero mode), then rows 1..N are packed
  float2* res = nullptr;
  float2* work = nullptr;
  PE_CUDA(p, cudaMallocAsync(reinterpret_cast<void**>(&res), sizeof(float2) * size_t(p->L) * count, p->stream));
  if (p->log2L > kMaxSmemLog2)
    PE_CUDA(p, cudaMallocAsync(reinterpret_cast<void**>(&work),
                               sizeof(float2) * sssp::large_work_elems(p->L) * size_t(count), p->stream));
  PE_CUDA(p, launch_dst_batch(p->log2L, reinterpret_cast<const float2*>(in), res, p->tabs, p->stream, work, count,
                              p->N, p->L, p->bc));
  PE_CUDA(p, cudaMemcpy2DAsync(out, sizeof(float2) * p->N, res + p->off, sizeof(float2) * p->L, sizeof(float2) * p->N,
                               count, cudaMemcpyDeviceToDevice, p->stream));
  PE_CUDA(p, cudaFreeAsync(res, p->stream));
  if (work) PE_CUDA(p, cudaFreeAsync(work, p->stream));
  return PE_OK;
}

pe_status pe_plan_set_kernel(pe_plan* p, int kernel) {
  if (!p) return PE_ERR_ARG;
  if (kernel != PE_KERNEL_AUTO && kernel != PE_KERNEL_CTA && kernel != PE_KERNEL_CLUSTER)
    return fail(p, PE_ERR_ARG, "kernel must be PE_KERNEL_AUTO, PE_KERNEL_CTA or PE_KERNEL_CLUSTER");
  if (kernel == PE_KERNEL_CLUSTER) {
    if (p->user_bc != PE_BC_DIRICHLET || !sssp_cluster::supported(p->log2L))
      return fail(p, PE_ERR_ARG, "the cluster kernel takes Dirichlet grids with N + 1 in [4096, 32768]");
    int a = 0, b = 0;
    PE_CUDA(p, sssp_cluster::max_active_clusters(p->log2L, false, &a));
    PE_CUDA(p, sssp_cluster::max_active_clusters(p->log2L, true, &b));
    if (a < 1 || b < 1) return fail(p, PE_ERR_ARG, "this device cannot hold a cluster of the required shape");
  }
  p->kernel = kernel;
  return PE_OK;
}

pe_status pe_plan_autotune(pe_plan* p, int steps, float* ms, int* chosen) {
  if (!p || steps < 1) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_plan_autotune");
  if (!p->field_set) return fail(p, PE_ERR_STATE, "pe_plan_autotune before pe_set_field");
  if (p->terms > 1 && p->nodes == 0) return fail(p, PE_ERR_STATE, "pe_plan_autotune with Neumann terms but no profile");
  int cands[2] = {PE_KERNEL_CTA, PE_KERNEL_CLUSTER};
  int ncand = 1;
  int clusters = 0;
  if (p->user_bc == PE_BC_DIRICHLET && sssp_cluster::supported(p->log2L) &&
      sssp_cluster::max_active_clusters(p->log2L, p->complex_profile, &clusters) == cudaSuccess && clusters > 0)
    ncand = 2;
  // the marcher's state and bookkeeping, restored after every trial
  std::vector<float> state(pe_state_size(p));
  double r_set = 0.0;
  long long steps_done = 0;
  pe_status st = pe_save_state(p, state.data(), &r_set, &steps_done);
  if (st != PE_OK) return st;
  const long long tl_rows = p->tl_rows;
  const std::vector<double> tl_ranges = p->tl_ranges;
  const int kernel0 = p->kernel;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PE_CUDA(p, cudaEventCreate(&e0));
  PE_CUDA(p, cudaEventCreate(&e1));
  float best = 0.f;
  int best_k = kernel0 == PE_KERNEL_AUTO ? PE_KERNEL_CTA : kernel0;
  for (int c = 0; c < ncand; ++c) {
    p->kernel = cands[c];
    float t = 0.f;
    for (int rep = 0; rep < 2 && st == PE_OK; ++rep) {  // the first run warms tables and caches
      PE_CUDA(p, cudaEventRecord(e0, p->stream));
      st = pe_march(p, steps);
      PE_CUDA(p, cudaEventRecord(e1, p->stream));
      if (st == PE_OK) st = check_status(p);
      if (st == PE_OK) PE_CUDA(p, cudaEventElapsedTime(&t, e0, e1));
      pe_status rs = pe_load_state(p, state.data(), r_set, steps_done);
      p->tl_rows = tl_rows;
      p->tl_ranges = tl_ranges;
      if (st == PE_OK) st = rs;
    }
    if (st != PE_OK) break;
    if (ms) ms[c] = t;
    if (c == 0 || t < best) {
      best = t;
      best_k = cands[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PE_OK) {
    p->kernel = kernel0;
    return st;
  }
  if (ncand < 2 && ms) ms[1] = -1.f;
  p->kernel = best_k;
  if (chosen) *chosen = best_k;
  return PE_OK;
}

pe_status pe_plan_set_operator(pe_plan* p, int op) {
  if (!p) return PE_ERR_ARG;
  if (op != PE_OP_SPECTRAL && op != PE_OP_FD3) return fail(p, PE_ERR_ARG, "op must be PE_OP_SPECTRAL or PE_OP_FD3");
  if (p->field_set || p->nodes > 0) return fail(p, PE_ERR_STATE, "set the operator before the profile and the field");
  if (op == PE_OP_FD3) {
    if (p->user_bc != PE_BC_DIRICHLET || !sssp_fd::supported(p->log2L))
      return fail(p, PE_ERR_ARG, "FD-SSP plans take Dirichlet grids with N + 1 in [8, 4096]");
    if (!p->dFDc) {
      std::vector<float4> c(2 * size_t(p->p));
      for (int j = 0; j < p->p; ++j) {
        const cd ab = p->pade.a[j] / p->pade.b[j];
        split_ff(ab, &c[2 * j]);
        split_ff(1.0 - ab, &c[2 * j + 1]);
      }
      PE_CUDA(p, cudaMalloc(&p->dFDc, sizeof(float4) * c.size()));
      PE_CUDA(p, cudaMemcpy(p->dFDc, c.data(), sizeof(float4) * c.size(), cudaMemcpyHostToDevice));
    }
  }
  p->op = op;
  return PE_OK;
}

pe_status pe_plan_set_shape(pe_plan* p, int points_per_thread) {
  if (!p) return PE_ERR_ARG;
  const int v = points_per_thread == 0 ? 8 : points_per_thread;
  if (v != 4 && v != 8 && v != 16) return fail(p, PE_ERR_ARG, "points_per_thread must be 0, 4, 8 or 16");
  if (v != 8 && (p->bc != PE_BC_DIRICHLET || !sssp_shapes::supported(p->log2L, v)))
    return fail(p, PE_ERR_ARG, "4 and 16 points per thread take Dirichlet grids with N + 1 in [256, 4096]");
  p->ppt = v;
  return PE_OK;
}

pe_status pe_plan_get_shape(const pe_plan* p, int* points_per_thread) {
  if (!p || !points_per_thread) return PE_ERR_ARG;
  *points_per_thread = (p->log2L <= kMaxSmemLog2 && !use_cluster(p, p->complex_profile)) ? shape_of(p) : 0;
  return PE_OK;
}

pe_status pe_plan_set_cluster_shape(pe_plan* p, int ncta, int push) {
  if (!p) return PE_ERR_ARG;
  if (push < -1 || push > 1) return fail(p, PE_ERR_ARG, "push must be -1 (default), 0 (pull) or 1 (push)");
  if (p->user_bc != PE_BC_DIRICHLET || !sssp_cluster::shape_supported(p->log2L, ncta, push))
    return fail(p, PE_ERR_ARG,
                "cluster shapes: Dirichlet grids with N + 1 in [4096, 32768]; ncta 0 (the size's default), "
                "8 (N + 1 <= 16384) or 16 (N + 1 >= 8192)");
  int a = 0, b = 0;
  PE_CUDA(p, sssp_cluster::max_active_clusters(p->log2L, false, &a, ncta, push));
  PE_CUDA(p, sssp_cluster::max_active_clusters(p->log2L, true, &b, ncta, push));
  if (a < 1 || b < 1) return fail(p, PE_ERR_ARG, "this device cannot hold a cluster of that shape");
  p->cl_ncta = ncta;
  p->cl_push = push;
  return PE_OK;
}

pe_status pe_plan_get_cluster_shape(const pe_plan* p, int* ncta, int* push) {
  if (!p || !ncta || !push) return PE_ERR_ARG;
  if (p->user_bc != PE_BC_DIRICHLET || !sssp_cluster::supported(p->log2L)) {
    *ncta = 0;
    *push = -1;
    return PE_OK;
  }
  cluster_shape_of(p, ncta, push);
  return PE_OK;
}

pe_status pe_plan_get_kernel(const pe_plan* p, int* kernel) {
  if (!p || !kernel) return PE_ERR_ARG;
  *kernel = use_cluster(p, p->complex_profile) ? PE_KERNEL_CLUSTER : PE_KERNEL_CTA;
  return PE_OK;
}

}  // extern "C"

namespace {

// The shapes the autotuners search, in the order of their timing outputs: one CTA at 4, 8 and
// 16 points per thread, then thread-block clusters of 8 CTAs (N + 1 = 4096 .. 16384) pulling
// and pushing the transform's exchange, then of 16 CTAs (N + 1 = 8192 .. 32768) pulling and
// pushing.
constexpr int kShapes = PE_AUTOTUNE_SHAPES;
const int kShapeKernel[kShapes] = {PE_KERNEL_CTA,     PE_KERNEL_CTA,     PE_KERNEL_CTA,    PE_KERNEL_CLUSTER,
                                   PE_KERNEL_CLUSTER, PE_KERNEL_CLUSTER, PE_KERNEL_CLUSTER};
const int kShapePpt[kShapes] = {4, 8, 16, 8, 8, 8, 8};
const int kShapeNcta[kShapes] = {0, 0, 0, 8, 8, 16, 16};
const int kShapePush[kShapes] = {-1, -1, -1, 0, 1, 0, 1};

bool shape_ok(const pe_plan* p, int c) {
  if (kShapeKernel[c] == PE_KERNEL_CLUSTER) {
    int clusters = 0;
    const int n = kShapeNcta[c];
    return p->user_bc == PE_BC_DIRICHLET && sssp_cluster::shape_supported(p->log2L, n, kShapePush[c]) &&
           sssp_cluster::max_active_clusters(p->log2L, p->complex_profile, &clusters, n, kShapePush[c]) ==
               cudaSuccess &&
           clusters > 0;
  }
  if (kShapePpt[c] == 8) return true;
  return p->bc == PE_BC_DIRICHLET && sssp_shapes::supported(p->log2L, kShapePpt[c]);
}

struct SavedMarch {
  std::vector<float> state;
  double r_set = 0.0;
  long long steps = 0, tl_rows = 0;
  std::vector<double> tl_ranges;
  int kernel = 0, ppt = 8, cl_ncta = 0, cl_push = -1;
};

pe_status save_march(pe_plan* p, SavedMarch* sv) {
  sv->state.resize(pe_state_size(p));
  pe_status st = pe_save_state(p, sv->state.data(), &sv->r_set, &sv->steps);
  sv->tl_rows = p->tl_rows;
  sv->tl_ranges = p->tl_ranges;
  sv->kernel = p->kernel;
  sv->ppt = p->ppt;
  sv->cl_ncta = p->cl_ncta;
  sv->cl_push = p->cl_push;
  return st;
}

pe_status restore_march(pe_plan* p, const SavedMarch& sv) {
  pe_status st = pe_load_state(p, sv.state.data(), sv.r_set, sv.steps);
  p->tl_rows = sv.tl_rows;
  p->tl_ranges = sv.tl_ranges;
  return st;
}

// Time `steps` range steps of the batch (a warm-up run, then a timed run) with every shape the
// plans can take, restoring their state after each run; set the fastest.
pe_status autotune_batch(pe_plan** plans, int count, int steps, float* ms, int* kernel, int* ppt) {
  pe_plan* p0 = plans[0];
  std::vector<SavedMarch> sv(static_cast<size_t>(count));
  for (int i = 0; i < count; ++i) {
    if (!plans[i]->field_set) return fail(p0, PE_ERR_STATE, "autotune before pe_set_field");
    if (plans[i]->terms > 1 && plans[i]->nodes == 0)
      return fail(p0, PE_ERR_STATE, "autotune with Neumann terms but no profile");
    pe_status st = save_march(plans[i], &sv[size_t(i)]);
    if (st != PE_OK) return st;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PE_CUDA(p0, cudaEventCreate(&e0));
  PE_CUDA(p0, cudaEventCreate(&e1));
  std::vector<int> st_steps(static_cast<size_t>(count), steps);
  float best = -1.f;
  int best_c = -1;
  pe_status st = PE_OK;
  for (int c = 0; c < kShapes && st == PE_OK; ++c) {
    bool any = false;
    for (int i = 0; i < count; ++i) any = any || shape_ok(plans[i], c);
    if (ms) ms[c] = -1.f;
    if (!any) continue;
    for (int i = 0; i < count; ++i)
      if (shape_ok(plans[i], c)) {
        plans[i]->kernel = kShapeKernel[c];
        plans[i]->ppt = kShapePpt[c];
        if (kShapeKernel[c] == PE_KERNEL_CLUSTER) {
          plans[i]->cl_ncta = kShapeNcta[c];
          plans[i]->cl_push = kShapePush[c];
        }
      }
    float t = 0.f;
    for (int rep = 0; rep < 2 && st == PE_OK; ++rep) {  // the first run warms tables and caches
      PE_CUDA(p0, cudaEventRecord(e0, p0->stream));
      st = pe_march_batch_steps(plans, st_steps.data(), count);
      PE_CUDA(p0, cudaEventRecord(e1, p0->stream));
      for (int i = 0; i < count && st == PE_OK; ++i) st = check_status(plans[i]);
      if (st == PE_OK) PE_CUDA(p0, cudaEventElapsedTime(&t, e0, e1));
      for (int i = 0; i < count; ++i) {
        pe_status rs = restore_march(plans[i], sv[size_t(i)]);
        if (st == PE_OK) st = rs;
      }
    }
    if (st != PE_OK) break;
    if (ms) ms[c] = t;
    if (best_c < 0 || t < best) {
      best = t;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < count; ++i) {  // the previous setting, then the winner where it applies
    plans[i]->kernel = sv[size_t(i)].kernel;
    plans[i]->ppt = sv[size_t(i)].ppt;
    plans[i]->cl_ncta = sv[size_t(i)].cl_ncta;
    plans[i]->cl_push = sv[size_t(i)].cl_push;
    if (st == PE_OK && best_c >= 0 && shape_ok(plans[i], best_c)) {
      plans[i]->kernel = kShapeKernel[best_c];
      plans[i]->ppt = kShapePpt[best_c];
      if (kShapeKernel[best_c] == PE_KERNEL_CLUSTER) {
        plans[i]->cl_ncta = kShapeNcta[best_c];
        plans[i]->cl_push = kShapePush[best_c];
      }
    }
  }
  if (st != PE_OK) return st;
  if (count > 1) {  // each solve's cost (transforms per step) on the chosen shape, for the launch order
    std::vector<unsigned long long> n0(static_cast<size_t>(count)), n1(static_cast<size_t>(count));
    for (int i = 0; i < count && st == PE_OK; ++i) st = pe_get_transform_count(plans[i], &n0[size_t(i)]);
    if (st == PE_OK) st = pe_march_batch_steps(plans, st_steps.data(), count);
    for (int i = 0; i < count && st == PE_OK; ++i) st = pe_get_transform_count(plans[i], &n1[size_t(i)]);
    for (int i = 0; i < count; ++i) {
      pe_status rs = restore_march(plans[i], sv[size_t(i)]);
      if (st == PE_OK) st = rs;
    }
    if (st != PE_OK) return st;
    for (int i = 0; i < count; ++i) plans[i]->cost = double(n1[size_t(i)] - n0[size_t(i)]) / double(steps);
  }
  if (kernel) *kernel = kShapeKernel[best_c];
  if (ppt) *ppt = kShapePpt[best_c];
  return PE_OK;
}

}  // namespace

extern "C" {

pe_status pe_plan_autotune_shapes(pe_plan* p, int steps, float* ms, int* kernel, int* points_per_thread) {
  if (!p || steps < 1) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_plan_autotune_shapes");
  return autotune_batch(&p, 1, steps, ms, kernel, points_per_thread);
}

pe_status pe_march_batch_autotune(pe_plan** plans, int count, int steps, float* ms, int* kernel,
                                  int* points_per_thread) {
  if (!plans || count < 1 || steps < 1) return PE_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!plans[i] || plans[i]->device != plans[0]->device) return PE_ERR_ARG;
  NvtxRange nvtx_("pe_march_batch_autotune");
  return autotune_batch(plans, count, steps, ms, kernel, points_per_thread);
}

size_t pe_state_size(const pe_plan* p) { return p ? 4 * size_t(p->L) : 0; }

pe_status pe_save_state(pe_plan* p, float* state, double* r_set, long long* steps) {
  if (!p || !state) return PE_ERR_ARG;
  if (!p->field_set) return fail(p, PE_ERR_STATE, "no field set");
  // spectral envelope, then its depth-domain copy (what pe_read_field reads)
  PE_CUDA(p, cudaMemcpyAsync(state, p->dYhat, sizeof(float2) * p->L, cudaMemcpyDeviceToHost, p->stream));
  PE_CUDA(p, cudaMemcpyAsync(state + 2 * size_t(p->L), p->dField, sizeof(float2) * p->L, cudaMemcpyDeviceToHost,
                             p->stream));
  if (r_set) *r_set = p->r_set;
  if (steps) *steps = p->steps_done;
  return check_status(p);
}

pe_status pe_load_state(pe_plan* p, const float* state, double r_set, long long steps) {
  if (!p || !state) return PE_ERR_ARG;
  if (steps < 0 || !std::isfinite(r_set)) return fail(p, PE_ERR_ARG, "steps must be >= 0 and r_set finite");
  PE_CUDA(p, cudaMemcpyAsync(p->dYhat, state, sizeof(float2) * p->L, cudaMemcpyHostToDevice, p->stream));
  PE_CUDA(p, cudaMemcpyAsync(p->dField, state + 2 * size_t(p->L), sizeof(float2) * p->L, cudaMemcpyHostToDevice,
                             p->stream));
  PE_CUDA(p, cudaMemsetAsync(p->dStatus, 0, sizeof(int), p->stream));
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  p->r_set = r_set;
  p->steps_done = steps;
  p->tl_rows = 0;
  p->tl_ranges.clear();
  p->field_set = true;
  return PE_OK;
}

pe_status pe_neumann_bound(pe_plan* p, int node, double* rho) {
  if (!p || !rho) return PE_ERR_ARG;
  if (node < 0 || node >= p->nodes) return fail(p, PE_ERR_ARG, "no such profile node");
  std::vector<float> v(p->L), vi;
  PE_CUDA(p, cudaMemcpyAsync(v.data(), p->dV + size_t(node) * p->L, sizeof(float) * p->L, cudaMemcpyDeviceToHost,
                             p->stream));
  if (p->complex_profile) {
    vi.resize(p->L);
    PE_CUDA(p, cudaMemcpyAsync(vi.data(), p->dVi + size_t(node) * p->L, sizeof(float) * p->L, cudaMemcpyDeviceToHost,
                               p->stream));
  }
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  double vmax = 0.0;
  for (int n = 0; n < p->L; ++n) vmax = std::max(vmax, std::hypot(double(v[n]), vi.empty() ? 0.0 : double(vi[n])));
  const bool periodic = (p->bc == PE_BC_PERIODIC);
  const double Hk = p->H;  // already the period 2H for Neumann plans
  for (int j = 0; j < p->p; ++j) {
    double mx = 0.0;
    for (int m = (periodic ? 0 : 1); m < p->L; ++m) {
      const double l = periodic ? double(m <= p->L / 2 ? m : m - p->L) : double(m);
      const double x = (periodic ? 2.0 : 1.0) * M_PI * l / (p->k0 * Hk);
      mx = std::max(mx, std::abs(p->pade.b[j] / (1.0 + p->pade.b[j] * (-x * x))));
    }
    rho[j] = vmax * mx;
  }
  return PE_OK;
}

pe_status pe_inject_status(pe_plan* p, int status) {
  if (!p) return PE_ERR_ARG;
  PE_CUDA(p, cudaMemcpyAsync(p->dStatus, &status, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  PE_CUDA(p, cudaStreamSynchronize(p->stream));
  return PE_OK;
}

pe_status pe_get_range(const pe_plan* p, double* r, long long* steps) {
  if (!p) return PE_ERR_ARG;
  if (r) *r = p->r_set + double(p->steps_done) * p->dr;
  if (steps) *steps = p->steps_done;
  return PE_OK;
}

}  // extern "C"
