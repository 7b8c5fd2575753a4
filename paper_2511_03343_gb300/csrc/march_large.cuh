// SSSP range march for grids larger than one CTA's shared memory (L = N + 1 = 8192 .. 65536).
//
// Same method as march_kernel.cuh (product-form Pade stages with hi/lo multipliers, Neumann
// series, spectral-resident field), but every length-L array lives in a per-solve workspace
// in global memory (L2-resident for a single solve, HBM for large batches), one CTA of 1024
// threads per solve, with a __syncthreads between passes (global writes are visible to the
// block after it).  The DST-I here is the scan-free form (two batched length-L FFTs, see
// dst_global): the prefix-scan form's odd outputs lose accuracy like sqrt(L) (3.6e-5 relative
// at L = 65536 in FP32), which these grids cannot afford.
// Element-wise work walks the natural index i = t + 1024 q, so every access is coalesced.
#pragma once
#include "march_kernel.cuh"

namespace sssp {

constexpr int kLargeNT = 1024;
constexpr int kLargeMinLog2 = 13;
constexpr int kLargeMaxLog2 = 16;

// workspace layout (float2 units): X (L) | W1 (2L) | W2 (2L) | acc (L) | t0 (L)
__host__ __device__ constexpr size_t large_work_elems(int L) { return 7 * size_t(L); }

template <int LOG2L>
struct CfgL {
  static constexpr int L = 1 << LOG2L;
  static constexpr int NT = kLargeNT;
  static constexpr int NW = NT / 32;
  static constexpr int PER = L / NT;        // elements per thread in element-wise loops
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

// One global-memory Stockham pass (radix R, span NS) over TWO independent length-L FFTs stored
// back to back (butterfly j < L/R belongs to the first, the rest to the second).
template <int LOG2L, int R, int NS>
__device__ __forceinline__ void gfft2_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                           const float2* __restrict__ tw) {
  constexpr int L = 1 << LOG2L, NB = L / R, PERB = 2 * NB / kLargeNT;
  constexpr int OFF = NS - 8;
  for (int q = 0; q < PERB; ++q) {
    const int jj = threadIdx.x + q * kLargeNT;
    const int h = (jj >= NB) ? L : 0;  // which of the two transforms
    const int j = jj - (h ? NB : 0);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[h + j + r * NB];
    const int k = j & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + OFF + (r - 1) * NS + k));
    dftR<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[h + base + r * NS] = v[r];
  }
}

template <int LOG2L, int NS>
__device__ __forceinline__ float2* gfft2_rest(float2* src, float2* dst, const float2* tw) {
  constexpr int L = 1 << LOG2L;
  if constexpr (NS >= L) {
    return src;
  } else {
    constexpr int R = (L / NS) >= 8 ? 8 : (L / NS);
    gfft2_pass<LOG2L, R, NS>(src, dst, tw);
    __syncthreads();
    return gfft2_rest<LOG2L, NS * R>(dst, src, tw);
  }
}

// Unnormalised DST-I of the L values in X (natural order, X[0] ignored), in place: on return
// X[m] = S_m (S_0 = 0).  W1, W2: 2L scratch each.  Scan-free (accurate) formulation of the
// odd extension's length-2L DFT after one radix-2 split:
//   S_{2k}   = (i/2) FFT_L(x_n - x_{L-n})_k,
//   S_{2k+1} = (i/2) FFT_L((x_n + x_{L-n}) e^{-i pi n/L})_k,   k < L/2,
// the two transforms run as one batched Stockham sequence.  On return all threads are past a
// barrier after the last write.
template <int LOG2L>
__device__ void dst_global(float2* X, float2* W1, float2* W2, const float2* __restrict__ tw,
                           const float* __restrict__ sinw) {
  constexpr int L = 1 << LOG2L;
  const int t = threadIdx.x;
  // first radix-8 pass (span 1) fused with the split into the two inputs; X -> W1
  for (int q = 0; q < (2 * (L / 8)) / kLargeNT; ++q) {
    const int jj = t + q * kLargeNT;
    const bool second = jj >= L / 8;
    const int j = second ? jj - L / 8 : jj;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int n = j + r * (L / 8);
      const float2 xn = (n == 0) ? make_float2(0.f, 0.f) : X[n];
      const float2 xm = (n == 0) ? make_float2(0.f, 0.f) : X[L - n];
      if (!second) {
        v[r] = xn - xm;
      } else {
        // e^{-i pi n/L} = cos - i sin, cos(pi n/L) from the sine table
        const float sn = __ldg(sinw + n);
        const float cs = (n <= L / 2) ? __ldg(sinw + (L / 2 - n)) : -__ldg(sinw + (n - L / 2));
        const float2 sm = xn + xm;
        v[r] = make_float2(fmaf(sm.x, cs, sm.y * sn), fmaf(sm.y, cs, -sm.x * sn));
      }
    }
    dft8(v);
    const int h = second ? L : 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) W1[h + 8 * j + r] = v[r];
  }
  __syncthreads();
  const float2* F = gfft2_rest<LOG2L, 8>(W1, W2, tw);
  for (int q = 0; q < (L / 2) / kLargeNT; ++q) {
    const int k = t + q * kLargeNT;
    const float2 fe = F[k];        // FFT of the differences
    const float2 fo = F[L + k];    // FFT of the weighted sums
    X[2 * k] = (k == 0) ? make_float2(0.f, 0.f) : make_float2(-0.5f * fe.y, 0.5f * fe.x);
    X[2 * k + 1] = make_float2(-0.5f * fo.y, 0.5f * fo.x);
  }
  __syncthreads();
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
  float2* const X = d.work;
  float2* const W1 = d.work + L;
  float2* const W2 = d.work + 3 * L;
  float2* const acc = d.work + 5 * L;
  float2* const t0 = d.work + 6 * L;
  const float out_scale = 2.0f / float(L);
  const bool iso = d.terms <= 1;
  const float tol2f = float(d.tol2);
  int status = kStatusOk;
  unsigned int ndst = 0;
  int nrec = 0;
  int node = d.node0;
  double next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
  const float* V = iso ? nullptr : d.V + (size_t)node * L;
  const float* Vi = (iso || d.Vi == nullptr) ? nullptr : d.Vi + (size_t)node * L;

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
        if (d.Vi != nullptr) Vi = d.Vi + (size_t)node * L;
      }
      for (int j = 0; j < d.p && status == kStatusOk; ++j) {
        const float2* Aj = d.A + (size_t)j * L;
        const float2* Bj = d.B + (size_t)j * L;
        for (int q = 0; q < C::PER; ++q) {
          const int i = t + q * kLargeNT;
          const float2 v = cmul(__ldg(Aj + i), y[i]);
          t0[i] = v;
          X[i] = v;
          acc[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        dst_global<LOG2L>(X, W1, W2, tw_g, sin_g);  // t_0 in depth space
        ++ndst;
        float first = 0.f;
        for (int m = 1; m < d.terms; ++m) {
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            X[i] = Vi ? cmul(make_float2(__ldg(V + i), __ldg(Vi + i)), X[i]) : __ldg(V + i) * X[i];
          }
          __syncthreads();
          dst_global<LOG2L>(X, W1, W2, tw_g, sin_g);  // DST(V t_{m-1})
          ++ndst;
          float nt = 0.f, nw = 0.f;
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            const float2 th = cmul(__ldg(Bj + i), X[i]);
            const float2 a = acc[i] + th;
            acc[i] = a;
            X[i] = th;
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
          dst_global<LOG2L>(X, W1, W2, tw_g, sin_g);  // t_m in depth space
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
        X[i] = out_scale * y[i];
      }
      __syncthreads();
      dst_global<LOG2L>(X, W1, W2, tw_g, sin_g);
      ++ndst;
      const float lr = float(10.0 * log10(d.r0 + double(s + 1) * d.dr));
      float* row = d.tl + (size_t)(d.rec0 + nrec) * d.N;
      for (int q = 0; q < C::PER; ++q) {
        const int n = t + q * kLargeNT;
        if (n >= 1) row[n - 1] = fmaf(-10.f, log10f(cabs2(X[n])), lr);
      }
      ++nrec;
      __syncthreads();
    }
  }
  // physical envelope for pe_read_field
  for (int q = 0; q < C::PER; ++q) {
    const int i = t + q * kLargeNT;
    X[i] = out_scale * y[i];
  }
  __syncthreads();
  dst_global<LOG2L>(X, W1, W2, tw_g, sin_g);
  ++ndst;
  for (int q = 0; q < C::PER; ++q) {
    const int i = t + q * kLargeNT;
    d.field[i] = X[i];
  }
  if (t == 0) {
    if (status != kStatusOk) atomicMax(d.status, status);
    atomicAdd(d.ndst, (unsigned long long)ndst);
  }
}

// One DST-I of a large grid: out = scale * DST(in); in holds N values, out L values.
// work: large_work_elems(L) float2 of scratch.
template <int LOG2L>
__global__ void __launch_bounds__(kLargeNT, 1)
    sssp_dst_large_kernel(const float2* __restrict__ in, float2* __restrict__ out, float scale, float2* work,
                          const float2* __restrict__ tw_g, const float* __restrict__ sin_g, long long in_stride = 0,
                          long long out_stride = 0) {
  constexpr int L = 1 << LOG2L;
  in += blockIdx.x * in_stride;
  out += blockIdx.x * out_stride;
  work += blockIdx.x * (long long)large_work_elems(L);
  float2* X = work;
  for (int n = threadIdx.x; n < L; n += kLargeNT) X[n] = (n == 0) ? make_float2(0.f, 0.f) : in[n - 1];
  __syncthreads();
  dst_global<LOG2L>(X, work + L, work + 3 * L, tw_g, sin_g);
  for (int n = threadIdx.x; n < L; n += kLargeNT) out[n] = scale * X[n];
}

}  // namespace sssp
