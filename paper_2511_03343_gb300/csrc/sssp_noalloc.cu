// pe_dst1_noalloc: the DST-I of pe_dst1 for callers that cannot allocate device memory.
//
// pe_dst1 stages its input and its length-L result in device memory the library allocates.
// Some callers cannot allow that: an application that reserves all of the GPU's memory for
// its own pool at start-up and forbids any later cudaMalloc (an allocation can fail under
// memory pressure, and the runtime may synchronise the device to serve it), or a plug-in
// that runs inside a host framework whose memory manager owns every device allocation.
// This entry point does the same work with its scratch in a fixed array compiled into the
// library, so a call allocates nothing.
//
// Limits and rules:
//  * N + 1 must be a power of two in [8, 4096] (the scratch holds two length-4096 complex
//    vectors: 64 KiB, plus 96 KiB of transform tables; every GPU that loads the library keeps
//    these arrays until the process exits).
//  * The first call on a device sets that device up (looks up the arrays' device addresses
//    and uploads the tables, synchronously).  Make that first call before any stream capture.
//    The set-up is tied to the device's current CUDA context: after cudaDeviceReset (which
//    reloads the arrays as zeros, possibly elsewhere) the next call sees a new context and
//    sets the device up again, so that call too must come before any capture.
//  * All calls share the one scratch array, which keeps the last call's contents.  Calls
//    whose work overlaps on the GPU (different streams, or several host threads) race on it;
//    order them on one stream or synchronise between them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/sssp.h"
#include "march_kernel.cuh"

namespace {

constexpr int kNoAllocMaxLog2 = 12;
constexpr int kNoAllocMaxL = 1 << kNoAllocMaxLog2;  // N <= 4095
constexpr int kNoAllocMinLog2 = 3;
constexpr int kMaxDevices = 64;

// scratch: [0, L) staged input (N values used), [kNoAllocMaxL, kNoAllocMaxL + L) transform output
static __device__ __align__(256) float2 g_noalloc_scratch[2 * kNoAllocMaxL];
// transform tables for every size L = 8..4096, the block of size L at offset L - 8
static __device__ __align__(256) float2 g_noalloc_tw[2 * kNoAllocMaxL];
static __device__ __align__(256) float g_noalloc_sin[2 * kNoAllocMaxL];

struct NoAllocDevice {
  bool ready = false;
  void* ctx = nullptr;        // the context the addresses and tables belong to
  float2* scratch = nullptr;  // device address of g_noalloc_scratch (host-side name is a stand-in)
  float2* tw = nullptr;
  float* sinw = nullptr;
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kMaxDevices];

// The calling thread's current context (driver API, looked up once through the runtime so
// the library needs no link against the driver library).
using CtxGetCurrentFn = int (*)(void**);
void* current_context() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

template <int LOG2L>
__global__ void __launch_bounds__(sssp::Cfg<LOG2L>::NT)
    sssp_noalloc_dst_kernel(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tw_g,
                            const float* __restrict__ sin_g) {
  using C = sssp::Cfg<LOG2L>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sssp::Smem<LOG2L> sm(smem_raw);
  const int t = threadIdx.x;
  sssp::load_tables<LOG2L>(sm.tw, sm.sinw, tw_g, sin_g);
  for (int n = t; n < C::L; n += C::NT) sm.bufA[sssp::pidx(n)] = (n == 0) ? make_float2(0.f, 0.f) : in[n - 1];
  __syncthreads();
  float2 o[8];
  sssp::dst_block<LOG2L>(sm.bufA, sm.bufB, sm.tw, sm.sinw, sm.scan_s, o);
  sssp::store8<LOG2L>(out + 8 * t, o);
}

template <int LOG2L>
cudaError_t noalloc_attr() {
  return cudaFuncSetAttribute(sssp_noalloc_dst_kernel<LOG2L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(sssp::Cfg<LOG2L>::SMEM));
}

template <int LOG2L>
cudaError_t noalloc_launch(const NoAllocDevice& d, cudaStream_t st) {
  constexpr int L = 1 << LOG2L;
  const float2* tw = d.tw + (L - 8);
  const float* sw = d.sinw + (L - 8);
  sssp_noalloc_dst_kernel<LOG2L><<<1, sssp::Cfg<LOG2L>::NT, sssp::Cfg<LOG2L>::SMEM, st>>>(
      d.scratch, d.scratch + kNoAllocMaxL, tw, sw);
  return cudaGetLastError();
}

cudaError_t noalloc_dispatch(int log2L, const NoAllocDevice& d, cudaStream_t st) {
  switch (log2L) {
    case 3: return noalloc_launch<3>(d, st);
    case 4: return noalloc_launch<4>(d, st);
    case 5: return noalloc_launch<5>(d, st);
    case 6: return noalloc_launch<6>(d, st);
    case 7: return noalloc_launch<7>(d, st);
    case 8: return noalloc_launch<8>(d, st);
    case 9: return noalloc_launch<9>(d, st);
    case 10: return noalloc_launch<10>(d, st);
    case 11: return noalloc_launch<11>(d, st);
    case 12: return noalloc_launch<12>(d, st);
  }
  return cudaErrorInvalidValue;
}

// Once per device, with that device current: device addresses of the file-scope arrays,
// the per-size tables (FP64 on the host, rounded once) and the kernels' shared-memory limit.
cudaError_t noalloc_setup(int dev, NoAllocDevice* out) {
  NoAllocDevice d;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.scratch), g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.tw), g_noalloc_tw);
  if (e != cudaSuccess) return e;
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.sinw), g_noalloc_sin);
  if (e != cudaSuccess) return e;
  std::vector<float2> tw(2 * kNoAllocMaxL, make_float2(0.f, 0.f));
  std::vector<float> sw(2 * kNoAllocMaxL, 0.f);
  for (int lg = kNoAllocMinLog2; lg <= kNoAllocMaxLog2; ++lg) {
    const int L = 1 << lg, off = L - 8;
    for (int q = 0; q < L; ++q) sw[off + q] = float(std::sin(M_PI * double(q) / double(L)));
    // Stockham twiddles exp(-2 pi i r k/(NS R)) of the passes after the first, at
    // (NS - 8) + (r - 1) NS + k within the size's block
    for (int ns = 8; ns < L; ns *= 8) {
      const int R = (L / ns) < 8 ? (L / ns) : 8;
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < ns; ++k) {
          const double ang = 2.0 * M_PI * double(r) * double(k) / (double(ns) * double(R));
          tw[off + (ns - 8) + (r - 1) * ns + k] = make_float2(float(std::cos(ang)), float(-std::sin(ang)));
        }
    }
  }
  e = cudaMemcpy(d.tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(d.sinw, sw.data(), sizeof(float) * sw.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  cudaError_t a[] = {noalloc_attr<3>(), noalloc_attr<4>(), noalloc_attr<5>(), noalloc_attr<6>(),
                     noalloc_attr<7>(), noalloc_attr<8>(), noalloc_attr<9>(), noalloc_attr<10>(),
                     noalloc_attr<11>(), noalloc_attr<12>()};
  for (cudaError_t x : a)
    if (x != cudaSuccess) return x;
  (void)dev;
  d.ready = true;
  *out = d;
  return cudaSuccess;
}

}  // namespace

extern "C" pe_status pe_dst1_noalloc(const float* in, float* out, int N, void* cuda_stream) {
  if (!in || !out) return PE_ERR_ARG;
  // range first, so that the power-of-two search below cannot overflow
  if (N < (1 << kNoAllocMinLog2) - 1 || N > kNoAllocMaxL - 1) return PE_ERR_ARG;
  int log2L = 0;
  while ((1 << log2L) < N + 1) ++log2L;
  if ((1 << log2L) != N + 1) return PE_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PE_ERR_CUDA;
  NoAllocDevice d;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice& cur = g_noalloc_dev[dev];
    if (!cur.ready || cur.ctx == nullptr || cur.ctx != current_context()) {
      cur.ready = false;
      if (noalloc_setup(dev, &cur) != cudaSuccess) return PE_ERR_CUDA;
      cur.ctx = current_context();  // the set-up's runtime calls made the context current
    }
    d = cur;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = sizeof(float2) * size_t(N);
  if (cudaMemcpyAsync(d.scratch, in, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return PE_ERR_CUDA;
  if (noalloc_dispatch(log2L, d, st) != cudaSuccess) return PE_ERR_CUDA;
  // the kernel writes all L output entries; entry 0 (the zero mode) is not returned
  if (cudaMemcpyAsync(out, d.scratch + kNoAllocMaxL + 1, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return PE_ERR_CUDA;
  return PE_OK;
}
