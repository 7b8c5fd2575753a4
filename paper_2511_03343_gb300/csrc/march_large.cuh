// SSSP range march for grids larger than one CTA's shared memory (L = N + 1 = 8192 .. 65536).
//
// Same method as march_kernel.cuh (product-form Pade stages with hi/lo multipliers, Neumann
// series, spectral-resident field), but every length-L array lives in a per-solve workspace
// in global memory (L2-resident for a single solve, HBM for large batches), one CTA of 512
// threads per solve, with a __syncthreads between passes (global writes are visible to the
// block after it).  The DST-I here is the DFT of the odd extension in two passes of
// shared-memory tiles (see dst_global), with no prefix scan: the scan form's odd outputs lose
// accuracy like sqrt(L) (3.6e-5 relative at L = 65536 in FP32), which these grids cannot afford.
// Element-wise work walks the natural index i = t + 512 q, so every access is coalesced.
#pragma once
#include "march_kernel.cuh"

namespace sssp {

constexpr int kLargeNT = 512;
constexpr int kLargeLog2Tile = 13;  // points per tile (16 per thread)
constexpr int kLargeTile = 1 << kLargeLog2Tile;
constexpr int kLargePT = kLargeTile / kLargeNT;  // points per thread per tile
constexpr int kLargeMinLog2 = 13;
constexpr int kLargeMaxLog2 = 16;

// workspace layout (float2 units): X (L) | W (2L) | w (L) | t0 (L)
__host__ __device__ constexpr size_t large_work_elems(int L) { return 5 * size_t(L); }

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

// A hint that moves the 128-byte line holding p into the L2 (no registers held; p is always an
// element of the arrays the pass reads).  Operands are fetched this way a tile before their
// register loads -- pass A: the sources of tile 1 before tile 0, of tile c + 2 during tile c;
// pass B: the sink operands of tile 0 before the pass, of tile + 1 during tile -- so those
// loads find their data in the L2 instead of waiting for HBM.
__device__ __forceinline__ void l2_prefetch(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Tables of the two-pass transform: per-pass Stockham twiddles of the P- and Q-point FFTs
// and w_{2L}^q, q in [0, 2L), each as a hi + lo pair of floats (float-float): a twiddle's
// FP32 representation error is the same in every transform, so it adds up coherently over
// the range steps; with the lo part every twiddle product carries only its own rounding.
struct LargeTabs {
  const float4* twP;
  const float4* twQ;
  const float4* tw2L;
};

// The DST-I of length N = L - 1 is the DFT of the odd extension z (length 2L: z_n = x_n,
// z_{2L-n} = -x_n, z_0 = z_L = 0): S_k = (i/2) Z_k, k in [1, L).  Four-step with 2L = P Q,
// n = Q n1 + n2, k = k1 + P k2:
//   pass A (columns n2): Y[k1][n2] = w_{2L}^{n2 k1} sum_{n1} z_{Q n1 + n2} w_P^{n1 k1}
//   pass B (rows k1):    Z_{k1 + P k2} = sum_{n2} Y[k1][n2] w_Q^{n2 k2},  only k2 < Q/2 kept.
// z being odd, column Q - n2 is column n2 negated with its rows reversed, so only the columns
// n2 in [0, Q/2] are transformed and stored (L + P values); pass B rebuilds the rest of a row
// from its partner row P - k1, and (Z being odd too) transforms only the rows k1 <= P/2, whose
// upper outputs are the partner rows' S values: half a 2L-point FFT in all.  Each pass moves tiles of 8192 points through shared memory
// (16 per thread); a transform reads x once, writes and reads the half intermediate once and
// writes S once: 32 B per point, the two global passes of 16 B per point.
template <int LOG2L>
struct BigCfg {
  static constexpr int L = 1 << LOG2L;
  static constexpr int LOG2P = (LOG2L + 1) / 2;
  static constexpr int LOG2Q = LOG2L + 1 - LOG2P;
  static constexpr int P = 1 << LOG2P, Q = 1 << LOG2Q;
  static constexpr int TILE = kLargeTile;
  static constexpr int LOG2TC = kLargeLog2Tile - LOG2P, LOG2TR = kLargeLog2Tile - LOG2Q;
  static constexpr int TC = 1 << LOG2TC, TR = 1 << LOG2TR;  // columns / rows per tile
  static constexpr int RSP = P + P / 16 + 1, RSQ = Q + Q / 16 + 1;  // padded FFT strides
  static constexpr int BUF = (TC * RSP > TR * RSQ) ? TC * RSP : TR * RSQ;
  // pass A's twiddles w_{2L}^e, e = col k1 < L, as the product of two table entries
  // w^{(e >> LOG2R) R} w^{e & (R - 1)}; pass B's w_Q^n, n < Q/2
  static constexpr int LOG2R = (LOG2L + 1) / 2;
  static constexpr int R = 1 << LOG2R, NT1 = L / R;
  // two tile buffers, the P- and Q-point twiddle tables, then the three tables above (all hi + lo)
  static constexpr size_t SMEM = sizeof(float2) * 2 * size_t(BUF) + sizeof(float4) * (P + Q + R + NT1 + Q / 2);
};

// Tile FFTs use radix-16 Stockham passes (radix min(16, F/NS) at span NS), one butterfly of 16
// points per thread.  Twiddles of the pass at span NS > 1: entry off(NS) + (r - 1) NS + k holds
// w^{r k / (NS RAD)}, off(NS) the entries of the earlier passes (the first pass needs none).
__host__ __device__ constexpr int large_rad(int F, int ns) { return (F / ns) >= 16 ? 16 : (F / ns); }
__host__ __device__ constexpr int large_twoff(int F, int NS) {
  int off = 0;
  for (int ns = 1; ns < NS; ns *= large_rad(F, ns))
    if (ns > 1) off += (large_rad(F, ns) - 1) * ns;
  return off;
}

// One Stockham pass (radix RAD, span NS) over the tile's independent FFTs of length 2^LOG2F,
// FFT f at shared offset f RS (padded index inside).
template <int LOG2F, int RS, int RAD, int NS>
__device__ __forceinline__ void tpass(const float2* __restrict__ src, float2* __restrict__ dst,
                                      const float4* __restrict__ tw) {  // tw in shared memory
  constexpr int F = 1 << LOG2F, NB = F / RAD, PER = (kLargeTile / RAD) / kLargeNT;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int jb = threadIdx.x + q * kLargeNT;
    const int f = jb / NB, jj = jb & (NB - 1);
    const float2* s = src + f * RS;
    float2 v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = s[pidx(jj + r * NB)];
    const int k = jj & (NS - 1);
    if constexpr (NS > 1) {
      constexpr int OFF = large_twoff(F, NS);
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = ffmul(tw[OFF + (r - 1) * NS + k], v[r]);
    }
    dftR<RAD>(v);
    float2* d = dst + f * RS;
    const int base = (jj - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) d[pidx(base + r * NS)] = v[r];
  }
}

// all passes of the tile's FFTs, src -> ...; returns the buffer holding the result
template <int LOG2F, int RS, int NS>
__device__ __forceinline__ float2* tfft(float2* src, float2* dst, const float4* tw) {
  constexpr int F = 1 << LOG2F;
  if constexpr (NS >= F) {
    return src;
  } else {
    constexpr int RAD = large_rad(F, NS);
    tpass<LOG2F, RS, RAD, NS>(src, dst, tw);
    __syncthreads();
    return tfft<LOG2F, RS, NS * RAD>(dst, src, tw);
  }
}

// copy the P- and Q-point twiddle tables behind the two tile buffers (once per kernel)
template <int LOG2L>
__device__ __forceinline__ void load_large_twiddles(float2* sm, const LargeTabs& tb) {
  using C = BigCfg<LOG2L>;
  float4* twP = reinterpret_cast<float4*>(sm + 2 * C::BUF);
  for (int i = threadIdx.x; i < C::P; i += kLargeNT) twP[i] = tb.twP[i];
  for (int i = threadIdx.x; i < C::Q; i += kLargeNT) twP[C::P + i] = tb.twQ[i];
  float4* tlo = twP + C::P + C::Q;  // w^e, e < R
  float4* thi = tlo + C::R;         // w^{i R}, i < L / R
  float4* tq = thi + C::NT1;        // w_Q^n = w_{2L}^{P n}, n < Q/2
  for (int i = threadIdx.x; i < C::R; i += kLargeNT) tlo[i] = tb.tw2L[i];
  for (int i = threadIdx.x; i < C::NT1; i += kLargeNT) thi[i] = tb.tw2L[i * C::R];
  for (int i = threadIdx.x; i < C::Q / 2; i += kLargeNT) tq[i] = tb.tw2L[C::P * i];
}

// Unnormalised DST-I S_k = sum_n x_n sin(pi n k/L), k in [0, L) (S_0 = 0), of the values the
// source gives: src(m, first) returns x_m (m in [1, L)); it is called twice per m in pass A (for
// z_m and z_{2L-m}), `first` true on the first.  The sink takes snk(k, S_k) once per k in pass B.
// Pass A reads every source value before pass B writes anything, so a source and sink may share
// an array (in-place transform).  W: 2L scratch.  On return all threads are past a barrier.
template <int LOG2L, class SRC, class SNK>
__device__ void dst_global(float2* W, const LargeTabs& tb, float2* sm, const SRC& src, SNK& snk) {
  using C = BigCfg<LOG2L>;
  constexpr int L = C::L, P = C::P, Q = C::Q, QH = Q / 2, QS = QH + 1;
  constexpr int TC = C::TC, TR = C::TR;
  constexpr int LOG2QH = C::LOG2Q - 1;
  constexpr int NA = QH / TC + 1;  // pass-A tiles; the last ends at column Q/2 (overlap rewrites)
  const int t = threadIdx.x;
  float2* bufA = sm;
  float2* bufB = sm + C::BUF;
  const float4* twP = reinterpret_cast<const float4*>(sm + 2 * C::BUF);  // copied by load_large_twiddles
  const float4* twQ = twP + P;
  const float4* tlo = twQ + Q;
  const float4* thi = tlo + C::R;
  const float4* tq = thi + C::NT1;
  constexpr int PT = kLargePT, PH = kLargePT / 2;
  float2 pre[PT + 1];
  // pass A: the P-point FFTs of the stored columns n2 in [0, Q/2], twiddled, into W[k1][n2]
  auto loadA = [&](int c) {
    const int cb = c < NA - 1 ? c * TC : QH - TC + 1;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int idx = t + q * kLargeNT;
      const int n1 = idx >> C::LOG2TC, col = cb + (idx & (TC - 1));
      const int n = Q * n1 + col;
      float2 z = make_float2(0.f, 0.f);
      if (n != 0 && n != L) {
        // a point of a self-mirrored column (0, Q/2) is visited twice, the others once
        const bool first = (n < L) || (col != 0 && col != QH);
        const float2 x = n < L ? src(n, first) : src(2 * L - n, first);
        z = n < L ? x : make_float2(-x.x, -x.y);
      }
      pre[q] = z;
    }
  };
  auto l2A = [&](int c2) {  // the 16-point lines of tile c2's sources, one line per thread
    constexpr int LPR = TC / 16;  // lines per row of the tile
    const int cb2 = c2 < NA - 1 ? c2 * TC : QH - TC + 1;
    const int n1 = t / LPR, col0 = cb2 + 16 * (t % LPR);
    int lo, hi;
    if (n1 < P / 2) {
      lo = Q * n1 + col0;
      hi = lo + 15;
    } else {
      hi = 2 * L - Q * n1 - col0;
      lo = hi - 15;
    }
    src.l2(lo < 1 ? 1 : lo);
    src.l2(hi > L - 1 ? L - 1 : hi);
  };
  if (NA > 1) l2A(1);
  loadA(0);
  for (int c = 0; c < NA; ++c) {
    const int cb = c < NA - 1 ? c * TC : QH - TC + 1;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int idx = t + q * kLargeNT;
      bufA[(idx & (TC - 1)) * C::RSP + pidx(idx >> C::LOG2TC)] = pre[q];
    }
    __syncthreads();
    if (c + 1 < NA) loadA(c + 1);
    if (c + 2 < NA) l2A(c + 2);
    const float2* F = tfft<C::LOG2P, C::RSP, 1>(bufA, bufB, twP);
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int idx = t + q * kLargeNT;
      const int k1 = idx >> C::LOG2TC, f = idx & (TC - 1);
      const int col = cb + f;
      const int e = col * k1;  // < L: col <= Q/2, k1 < P
      W[k1 * QS + col] = ffmul(thi[e >> C::LOG2R], ffmul(tlo[e & (C::R - 1)], F[f * C::RSP + pidx(k1)]));
    }
    __syncthreads();
  }
  // pass B: the rows k in [0, P/2].  The odd symmetry of z gives the unstored half of a row from
  // its partner row P - k: Y[k][Q - n] = -w_Q^{-n} Y[P - k][n] (k != 0), -Y[0][n] (k = 0).  A row's
  // Q outputs are Z_{k + P k2}; those with k + P k2 >= L are -Z at 2L - k - P k2 = (P - k) +
  // P (Q - 1 - k2), the partner row's, so one FFT per row pair yields both rows' S values
  // (rows 0 and P/2 are their own partners: only their first Q/2 outputs are kept).
  constexpr int NBT = (P / 2) / TR + 1;  // the last tile ends at row P/2 (its other rows: done)
  auto rowof = [&](int tile, int sl) { return (tile < NBT - 1 ? tile * TR : P / 2 - TR + 1) + sl; };
  auto l2B = [&](int tile) {  // the lines of a tile's sink operands, one per thread
    constexpr int LPK = TR / 16;          // lines per output column k2 and side
    constexpr int NL1 = (Q / 2) * LPK;    // lines per side (own rows, partner rows)
    const int side = t / NL1, i = t % NL1, j2 = i / LPK;
    const int k0 = rowof(tile, 16 * (i % LPK));
    int lo, hi;
    if (side == 0) {
      lo = k0 + P * j2;
      hi = lo + 15;
    } else {
      hi = P - k0 + P * j2;
      lo = hi - 15;
    }
    snk.l2(lo < 0 ? 0 : lo);
    snk.l2(hi > L - 1 ? L - 1 : hi);
  };
  if (SNK::kL2) l2B(0);
  auto loadB = [&](int tile) {
#pragma unroll
    for (int q = 0; q < PH; ++q) {  // own stored half, columns [0, Q/2)
      const int idx = t + q * kLargeNT;
      pre[q] = W[rowof(tile, idx >> LOG2QH) * QS + (idx & (QH - 1))];
    }
#pragma unroll
    for (int q = 0; q < PH; ++q) {  // the partner's stored columns [1, Q/2) (column 0 unused)
      const int idx = t + q * kLargeNT;
      const int k = rowof(tile, idx >> LOG2QH);
      pre[PH + q] = W[((P - k) & (P - 1)) * QS + (idx & (QH - 1))];
    }
    if (t < TR) pre[PT] = W[rowof(tile, t) * QS + QH];
  };
  // output slot q of this thread: its target index, or false where another slot has it
  auto target = [&](int tile, int q, int& tgt, bool& neg) {
    const int idx = t + q * kLargeNT;
    const int k2 = idx >> C::LOG2TR, k = rowof(tile, idx & (TR - 1));
    if (tile == NBT - 1 && k != P / 2) return false;
    const int kap = k + P * k2;
    if (kap < L) {
      tgt = kap;
      neg = false;
      return true;
    }
    if (k == 0 || k == P / 2) return false;
    tgt = 2 * L - kap;
    neg = true;
    return true;
  };
  loadB(0);
  for (int tile = 0; tile < NBT; ++tile) {
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      const int idx = t + q * kLargeNT;
      const int sl = idx >> LOG2QH, n = idx & (QH - 1);
      bufA[sl * C::RSQ + pidx(n)] = pre[q];
      if (n != 0) {  // Y[k][Q - n] from the partner row
        float2 r = make_float2(-pre[PH + q].x, -pre[PH + q].y);
        if (rowof(tile, sl) != 0) {  // times w_Q^{-n} = conj(w_{2L}^{P n})
          const float4 w = tq[n];
          r = ffmul(make_float4(w.x, -w.y, w.z, -w.w), r);
        }
        bufA[sl * C::RSQ + pidx(Q - n)] = r;
      }
    }
    if (t < TR) bufA[t * C::RSQ + pidx(QH)] = pre[PT];
    __syncthreads();
    // the sink's operands for the first half of this tile's outputs, and the next tile, load
    // during the FFT
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      int tg;
      bool ng;
      if (target(tile, q, tg, ng)) snk.prefetch(q, tg);
    }
    if (tile + 1 < NBT) loadB(tile + 1);
    if (SNK::kL2 && tile + 1 < NBT) l2B(tile + 1);
    const float2* F = tfft<C::LOG2Q, C::RSQ, 1>(bufA, bufB, twQ);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      if (half == 1) {
#pragma unroll
        for (int q = 0; q < PH; ++q) {
          int tg;
          bool ng;
          if (target(tile, PH + q, tg, ng)) snk.prefetch(q, tg);
        }
      }
#pragma unroll
      for (int q = 0; q < PH; ++q) {
        int tg;
        bool ng;
        if (target(tile, half * PH + q, tg, ng)) {
          const int idx = t + (half * PH + q) * kLargeNT;
          const float2 zk = F[(idx & (TR - 1)) * C::RSQ + pidx(idx >> C::LOG2TR)];
          const float2 sv = ng ? make_float2(0.5f * zk.y, -0.5f * zk.x) : make_float2(-0.5f * zk.y, 0.5f * zk.x);
          snk.put(q, tg, (tg == 0) ? make_float2(0.f, 0.f) : sv);
        }
      }
    }
    __syncthreads();
  }
}

// sources (depth or spectral values the transform reads) and sinks (where its outputs go)
struct SrcArr {  // x_m = a[m]
  const float2* a;
  __device__ __forceinline__ float2 operator()(int m, bool) const { return a[m]; }
  __device__ __forceinline__ void l2(int m) const { l2_prefetch(a + m); }
};
struct SrcV {  // x_m = V_m a[m] (V real, or V + i Vi)
  const float2* a;
  const float* V;
  const float* Vi;
  __device__ __forceinline__ float2 operator()(int m, bool) const {
    const float2 x = a[m];
    return Vi ? cmul(make_float2(__ldg(V + m), __ldg(Vi + m)), x) : __ldg(V + m) * x;
  }
  __device__ __forceinline__ void l2(int m) const {
    l2_prefetch(a + m);
    l2_prefetch(V + m);
    if (Vi) l2_prefetch(Vi + m);
  }
};
struct SrcStage {  // x_m = t0_m = A_m y_m; on the first visit also t0[m] = w[m] = x_m
  const float2* A;
  const float2* y;
  float2* t0;
  float2* w;
  __device__ __forceinline__ float2 operator()(int m, bool first) const {
    const float2 v = cmul(__ldg(A + m), y[m]);
    if (first) {
      t0[m] = v;
      w[m] = v;
    }
    return v;
  }
  __device__ __forceinline__ void l2(int m) const {
    l2_prefetch(A + m);
    l2_prefetch(y + m);
  }
};
struct SrcScaled {  // x_m = s y_m
  const float2* y;
  float s;
  __device__ __forceinline__ float2 operator()(int m, bool) const { return s * y[m]; }
  __device__ __forceinline__ void l2(int m) const { l2_prefetch(y + m); }
};
// A sink takes put(q, k, S_k) for its q-th output of a tile; prefetch(q, k) is called for the
// same (q, k) before the tile's FFT, so a sink can load its own operands early.
struct SnkArr {
  static constexpr bool kL2 = false;  // write-only: no operands to fetch
  float2* a;
  __device__ __forceinline__ void l2(int) {}
  __device__ __forceinline__ void prefetch(int, int) {}
  __device__ __forceinline__ void put(int, int k, float2 v) { a[k] = v; }
};
// The partial sum w_j = t_0 + t_1 + .. is kept itself (not t_1 + .. beside t_0), so a term
// streams B and w, and the stage's combine reads t_0 once: y <- R y + beta (w - t_0).
struct SnkTerm {  // t_m = B_k S_k: w += t_m, X = t_m, and the norm partials of the stop test
  static constexpr bool kL2 = true;
  __device__ __forceinline__ void l2(int k) {
    l2_prefetch(B + k);
    l2_prefetch(w + k);
  }
  const float2* B;
  float2* w;
  float2* X;
  float nt, nw;
  float2 pb[kLargePT / 2], pw[kLargePT / 2];  // B and w of the tile's outputs
  __device__ __forceinline__ void prefetch(int q, int k) {
    pb[q] = __ldg(B + k);
    pw[q] = w[k];
  }
  __device__ __forceinline__ void put(int q, int k, float2 v) {
    if (k == 0) {  // the zero mode: t_m = 0, w[0] and t0[0] stay 0
      X[0] = make_float2(0.f, 0.f);
      return;
    }
    const float2 th = cmul(pb[q], v);
    const float2 a = pw[q] + th;
    w[k] = a;
    X[k] = th;
    nt += cabs2(th);
    nw += cabs2(a);
  }
};
struct SnkTL {  // TL row: -10 log10 |u_n|^2 + 10 log10 r, n = 1..N
  static constexpr bool kL2 = false;
  float* row;
  float lr;
  __device__ __forceinline__ void l2(int) {}
  __device__ __forceinline__ void prefetch(int, int) {}
  __device__ __forceinline__ void put(int, int k, float2 v) {
    if (k >= 1) row[k - 1] = fmaf(-10.f, log10f(cabs2(v)), lr);
  }
};

template <int LOG2L>
__global__ void __launch_bounds__(kLargeNT, 1)
    sssp_march_large_kernel(const SolveDesc* __restrict__ descs, const LargeTabs tb) {
  using C = CfgL<LOG2L>;
  constexpr int L = C::L;
  extern __shared__ __align__(16) float2 tile_smem[];
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
  float2* const W = d.work + L;
  float2* const wsum = d.work + 3 * L;  // w_j = t_0 + t_1 + .. (spectral)
  float2* const t0 = d.work + 4 * L;
  const float out_scale = 2.0f / float(L);
  const bool iso = d.terms <= 1;
  const float tol2f = float(d.tol2);  // the FP32 prefilter of the FP64 stop test
  int status = kStatusOk;
  unsigned int ndst = 0;
  int nrec = 0;
  int node = d.node0;
  double next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
  const float* V = iso ? nullptr : d.V + (size_t)node * L;
  const float* Vi = (iso || d.Vi == nullptr) ? nullptr : d.Vi + (size_t)node * L;
  if (t == 0) {  // the zero mode is never visited by the transform's source
    wsum[0] = make_float2(0.f, 0.f);
    t0[0] = make_float2(0.f, 0.f);
  }
  load_large_twiddles<LOG2L>(tile_smem, tb);
  __syncthreads();

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
        // t_0 = L_j^{-1} y in depth space; the source also sets t0 and w = t0 (spectral)
        {
          SnkArr sk{X};
          dst_global<LOG2L>(W, tb, tile_smem, SrcStage{d.A + (size_t)j * L, y, t0, wsum}, sk);
        }
        ++ndst;
        float first = 0.f;
        for (int m = 1; m < d.terms; ++m) {
          SnkTerm sk{d.B + (size_t)j * L, wsum, X, 0.f, 0.f, {}, {}};
          dst_global<LOG2L>(W, tb, tile_smem, SrcV{X, V, Vi}, sk);  // B DST(V t_{m-1}), w += t_m
          ++ndst;
          const float snt = block_sum<LOG2L>(sk.nt, red);
          const float snw = block_sum<LOG2L>(sk.nw, red + C::NW);
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
          if (neumann_stop_fast(snt, snw, d.tol2, tol2f)) break;
          SnkArr sx{X};
          dst_global<LOG2L>(W, tb, tile_smem, SrcArr{X}, sx);  // t_m in depth space
          ++ndst;
        }
        {
          const float4* rp = d.R + (size_t)j * L;
          const float2 bj = d.beta[j];
#pragma unroll 4
          for (int q = 0; q < C::PER; ++q) {
            const int i = t + q * kLargeNT;
            y[i] = ffmul(__ldg(rp + i), y[i]) + cmul(bj, wsum[i] - t0[i]);
          }
        }
        __syncthreads();
      }
      if (status != kStatusOk) break;
    }
    const long long gs = d.step0 + s + 1;
    if (d.tl_every > 0 && gs % d.tl_every == 0) {
      const float lr = float(10.0 * log10(d.r0 + double(s + 1) * d.dr));
      SnkTL sk{d.tl + (size_t)(d.rec0 + nrec) * d.N, lr};
      dst_global<LOG2L>(W, tb, tile_smem, SrcScaled{y, out_scale}, sk);
      ++ndst;
      ++nrec;
    }
  }
  {  // physical envelope for pe_read_field
    SnkArr sk{d.field};
    dst_global<LOG2L>(W, tb, tile_smem, SrcScaled{y, out_scale}, sk);
    ++ndst;
  }
  if (t == 0) {
    if (status != kStatusOk) atomicMax(d.status, status);
    atomicAdd(d.ndst, (unsigned long long)ndst);
  }
}

// One DST-I of a large grid: out = scale * DST(in); in holds N values, out L values.
// work: large_work_elems(L) float2 of scratch (2L used).
struct SrcIn {  // x_m = in[m - 1]
  const float2* in;
  __device__ __forceinline__ float2 operator()(int m, bool) const { return in[m - 1]; }
  __device__ __forceinline__ void l2(int m) const { l2_prefetch(in + m - 1); }
};
struct SnkScaled {
  static constexpr bool kL2 = false;
  float2* out;
  float s;
  __device__ __forceinline__ void l2(int) {}
  __device__ __forceinline__ void prefetch(int, int) {}
  __device__ __forceinline__ void put(int, int k, float2 v) { out[k] = s * v; }
};

template <int LOG2L>
__global__ void __launch_bounds__(kLargeNT, 1)
    sssp_dst_large_kernel(const float2* __restrict__ in, float2* __restrict__ out, float scale, float2* work,
                          const LargeTabs tb, long long in_stride = 0, long long out_stride = 0) {
  extern __shared__ __align__(16) float2 tile_smem[];
  in += blockIdx.x * in_stride;
  out += blockIdx.x * out_stride;
  work += blockIdx.x * (long long)large_work_elems(1 << LOG2L);
  load_large_twiddles<LOG2L>(tile_smem, tb);
  __syncthreads();
  SnkScaled sk{out, scale};
  dst_global<LOG2L>(work, tb, tile_smem, SrcIn{in}, sk);
}

}  // namespace sssp
