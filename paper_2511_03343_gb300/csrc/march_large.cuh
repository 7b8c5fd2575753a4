// SSSP range march for grids larger than one CTA's shared memory (L = N + 1 = 8192 .. 65536).
//
// Same method and arithmetic as march_kernel.cuh (product-form Pade stages, Neumann series,
// DST-I via one complex FFT of length L with sine pre-weighting, pair post-processing and a
// prefix scan), but every length-L array lives in a per-solve workspace in global memory
// (L2-resident for a single solve, HBM for large batches): the FFT is a sequence of
// radix-8 Stockham passes through global memory, one CTA of 1024 threads per solve, with a
// __syncthreads between passes (global writes are visible to the block after it).
// Element-wise work walks the natural index i = t + 1024 q, so every access is coalesced.
#pragma once
#include "march_kernel.cuh"

namespace sssp {

constexpr int kLargeNT = 1024;
constexpr int kLargeMinLog2 = 13;
constexpr int kLargeMaxLog2 = 16;

// workspace layout (float2 units): bufA | bufB | acc | t0, each L long
__host__ __device__ constexpr size_t large_work_elems(int L) { return 4 * size_t(L); }

template <int LOG2L>
struct CfgL {
  static constexpr int L = 1 << LOG2L;
  static constexpr int NT = kLargeNT;
  static constexpr int NW = NT / 32;
  static constexpr int PER = L / NT;        // elements per thread in element-wise loops
  static constexpr int CH = (L / 2) / NT;   // scan chunk (k values) per thread
};

// block sum of one float; every thread gets the same total (red: NW floats of shared memory)
template <int LOG2L>
__device__ __forceinline__ float block_sum(float v, float* red) {
  using C = CfgL<LOG2L>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // previous users of red are done
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = (lane < C::NW) ? red[lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One global-memory Stockham pass (radix R, span NS), butterflies j = t + NT q.
template <int LOG2L, int R, int NS>
__device__ __forceinline__ void gfft_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                          const float2* __restrict__ tw) {
  constexpr int L = 1 << LOG2L, NB = L / R, PERB = NB / kLargeNT;
  constexpr int OFF = NS - 8;
  for (int q = 0; q < PERB; ++q) {
    const int j = threadIdx.x + q * kLargeNT;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * NB];
    const int k = j & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + OFF + (r - 1) * NS + k));
    dftR<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * NS] = v[r];
  }
}

template <int LOG2L, int NS>
__device__ __forceinline__ float2* gfft_rest(float2* src, float2* dst, const float2* tw) {
  constexpr int L = 1 << LOG2L;
  if constexpr (NS >= L) {
    return src;
  } else {
    constexpr int R = (L / NS) >= 8 ? 8 : (L / NS);
    gfft_pass<LOG2L, R, NS>(src, dst, tw);
    __syncthreads();
    return gfft_rest<LOG2L, NS * R>(dst, src, tw);
  }
}

// Unnormalised DST-I of the L values in `a` (natural order, a[0] ignored), result S_m in natural
// order in the returned buffer (a or b; S_0 = 0).  `b` is scratch.  On return all threads are
// past a barrier after the last write.
template <int LOG2L>
__device__ float2* dst_global(float2* a, float2* b, const float2* __restrict__ tw, const float* __restrict__ sinw,
                              float* red) {
  using C = CfgL<LOG2L>;
  constexpr int L = C::L;
  const int t = threadIdx.x;
  // first radix-8 pass (span 1) fused with the sine pre-weighting; a -> b
  for (int q = 0; q < (L / 8) / kLargeNT; ++q) {
    const int j = t + q * kLargeNT;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int n = j + r * (L / 8);
      const float2 xn = a[n];
      const float2 xm = a[(L - n) & (L - 1)];
      const float s = __ldg(sinw + n);
      v[r] = make_float2(fmaf(s, xn.x + xm.x, 0.5f * (xn.x - xm.x)), fmaf(s, xn.y + xm.y, 0.5f * (xn.y - xm.y)));
    }
    dft8(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) b[8 * j + r] = v[r];
  }
  __syncthreads();
  float2* F = gfft_rest<LOG2L, 8>(b, a, tw);
  float2* O = (F == a) ? b : a;
  // post-processing over the thread's chunk k in [t CH, (t+1) CH): even outputs from the pairs,
  // odd outputs S_{2k+1} = sum_{k' <= k} D_{k'} by a local sum + block exclusive scan
  float2 tot = make_float2(0.f, 0.f);
  const int k0 = t * C::CH;
  for (int c = 0; c < C::CH; ++c) {
    const int k = k0 + c;
    const float2 yk = F[k];
    const float2 ym = F[(L - k) & (L - 1)];
    tot = tot + ((k == 0) ? 0.5f * yk : 0.5f * (yk + ym));
  }
  // exclusive scan of the thread totals
  const int lane = t & 31, warp = t >> 5;
  float2 inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float nx = __shfl_up_sync(0xffffffffu, inc.x, o);
    const float ny = __shfl_up_sync(0xffffffffu, inc.y, o);
    if (lane >= o) inc = inc + make_float2(nx, ny);
  }
  float2* wsum = reinterpret_cast<float2*>(red);  // NW float2
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  float2 off = make_float2(0.f, 0.f);
  for (int w = 0; w < warp; ++w) off = off + wsum[w];
  float2 run = off + inc - tot;  // exclusive prefix of this thread's chunk
  for (int c = 0; c < C::CH; ++c) {
    const int k = k0 + c;
    const float2 yk = F[k];
    const float2 ym = F[(L - k) & (L - 1)];
    run = run + ((k == 0) ? 0.5f * yk : 0.5f * (yk + ym));
    O[2 * k] = make_float2(-0.5f * (yk.y - ym.y), 0.5f * (yk.x - ym.x));
    O[2 * k + 1] = run;
  }
  __syncthreads();
  return O;
}

template <int LOG2L>
__global__ void __launch_bounds__(kLargeNT, 1)
    sssp_march_large_kernel(const SolveDesc* __restrict__ descs, const float2* __restrict__ tw_g,
                            const float* __restrict__ sin_g) {
  using C = CfgL<LOG2L>;
  constexpr int L = C::L;
  __shared__ SolveDesc d;
  __shared__ float red[2 * C::NW];
  const int t = threadIdx.x;
  {
    const int* src = reinterpret_cast<const int*>(descs + blockIdx.x);
    int* dst = reinterpret_cast<int*>(&d);
    for (int i = t; i < int(sizeof(SolveDesc) / sizeof(int)); i += kLargeNT) dst[i] = src[i];
  }
  __syncthreads();
  float2* const y = d.yhat;
  float2* const bufA = d.work;
  float2* const bufB = d.work + L;
  float2* const acc = d.work + 2 * L;
  float2* const t0 = d.work + 3 * L;
  const float out_scale = 2.0f / float(L);
  const bool iso = d.terms <= 1;
  const float tol2f = float(d.tol2);
  int status = kStatusOk;
  unsigned int ndst = 0;
  int nrec = 0;
  int node = d.node0;
  double next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
  const float* V = iso ? nullptr : d.V + (size_t)node * L;

  for (int s = 0; s < d.steps && status == kStatusOk; ++s) {
    if (iso) {
      for (int q = 0; q < C::PER; ++q) {
        const int i = t + q * kLargeNT;
        y[i] = ffmul(__ldg(d.G + i), y[i]);
      }
      __syncthreads();
    } else {
      const double rmid = d.r0 + (double(s) + 0.5) * d.dr;
      if (rmid >= next_r) {
        while (node + 1 < d.nodes && d.node_r[node + 1] <= rmid) ++node;
        next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
        V = d.V + (size_t)node * L;
      }
      for (int j = 0; j < d.p && status == kStatusOk; ++j) {
        const float2* Aj = d.A + (size_t)j * L;
        const float2* Bj = d.B + (size_t)j * L;
        for (int q = 0; q < C::PER; ++q) {
          const int i = t + q * kLargeNT;
          const float2 v = cmul(__ldg(Aj + i), y[i]);
          t0[i] = v;
          bufA[i] = v;
          acc[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2* tp = dst_global<LOG2L>(bufA, bufB, tw_g, sin_g, red);  // t_0 in depth space
        ++ndst;
        float first = 0.f;
        for (int m = 1; m < d.terms; ++m) {
          float2* other = (tp == bufA) ? bufB : bufA;
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            tp[i] = __ldg(V + i) * tp[i];
          }
          __syncthreads();
          float2* sh = dst_global<LOG2L>(tp, other, tw_g, sin_g, red);  // DST(V t_{m-1})
          ++ndst;
          float nt = 0.f, nw = 0.f;
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            const float2 th = cmul(__ldg(Bj + i), sh[i]);
            const float2 a = acc[i] + th;
            acc[i] = a;
            sh[i] = th;
            nt += cabs2(th);
            nw += cabs2(t0[i] + a);
          }
          const float snt = block_sum<LOG2L>(nt, red);
          const float snw = block_sum<LOG2L>(nw, red + C::NW);
          if (m == d.terms - 1) break;
          if (!isfinite(snt) || !isfinite(snw)) {
            status = kStatusNumeric;
            break;
          }
          if (m == 1) first = snt;
          else if (first > 0.f && snt > 1e8f * first) {
            status = kStatusDiverged;
            break;
          }
          if (snt <= tol2f * snw) break;
          tp = dst_global<LOG2L>(sh, (sh == bufA) ? bufB : bufA, tw_g, sin_g, red);  // t_m in depth space
          ++ndst;
        }
        {
          const float4* rp = d.R + (size_t)j * L;
          const float2 bj = d.beta[j];
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            y[i] = ffmul(__ldg(rp + i), y[i]) + cmul(bj, acc[i]);
          }
        }
        __syncthreads();
      }
      if (status != kStatusOk) break;
    }
    const long long gs = d.step0 + s + 1;
    if (d.tl_every > 0 && gs % d.tl_every == 0) {
      for (int q = 0; q < C::PER; ++q) {
        const int i = t + q * kLargeNT;
        bufA[i] = out_scale * y[i];
      }
      __syncthreads();
      float2* u = dst_global<LOG2L>(bufA, bufB, tw_g, sin_g, red);
      ++ndst;
      const float lr = float(10.0 * log10(d.r0 + double(s + 1) * d.dr));
      float* row = d.tl + (size_t)(d.rec0 + nrec) * d.N;
      for (int q = 0; q < C::PER; ++q) {
        const int n = t + q * kLargeNT;
        if (n >= 1) row[n - 1] = fmaf(-10.f, log10f(cabs2(u[n])), lr);
      }
      ++nrec;
      __syncthreads();
    }
  }
  // physical envelope for pe_read_field
  for (int q = 0; q < C::PER; ++q) {
    const int i = t + q * kLargeNT;
    bufA[i] = out_scale * y[i];
  }
  __syncthreads();
  float2* u = dst_global<LOG2L>(bufA, bufB, tw_g, sin_g, red);
  ++ndst;
  for (int q = 0; q < C::PER; ++q) {
    const int i = t + q * kLargeNT;
    d.field[i] = u[i];
  }
  if (t == 0) {
    if (status != kStatusOk) atomicMax(d.status, status);
    atomicAdd(d.ndst, (unsigned long long)ndst);
  }
}

// One DST-I of a large grid: out = scale * DST(in); in holds N values, out L values.
// work: 2 L float2 of scratch.
template <int LOG2L>
__global__ void __launch_bounds__(kLargeNT, 1)
    sssp_dst_large_kernel(const float2* __restrict__ in, float2* __restrict__ out, float scale, float2* work,
                          const float2* __restrict__ tw_g, const float* __restrict__ sin_g) {
  constexpr int L = 1 << LOG2L;
  __shared__ float red[2 * CfgL<LOG2L>::NW];
  float2* a = work;
  float2* b = work + L;
  for (int n = threadIdx.x; n < L; n += kLargeNT) a[n] = (n == 0) ? make_float2(0.f, 0.f) : in[n - 1];
  __syncthreads();
  float2* r = dst_global<LOG2L>(a, b, tw_g, sin_g, red);
  for (int n = threadIdx.x; n < L; n += kLargeNT) out[n] = scale * r[n];
}

}  // namespace sssp
