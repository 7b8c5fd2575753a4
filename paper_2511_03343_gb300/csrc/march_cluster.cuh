// SSSP range march of ONE solve spread over a thread-block cluster of NCTA CTAs (NCTA = 8 or
// 16, one CTA per SM), every length-L array held in the cluster's distributed shared memory.
//
// The per-step algorithm is the one of march_kernel.cuh (product form, Eq. Neumann); what
// changes is how a DST-I of length N = L - 1 is laid out over the cluster.
//
// Transform (scan-free form, unnormalised, x_0 = 0):
//   u_n = x_n - x_{L-n},  v_n = (x_n + x_{L-n}) e^{-i pi n/L},   n in [0, L)
//   S_{2k} = (i/2) FFT_L(u)_k,  S_{2k+1} = (i/2) FFT_L(v)_k,       k in [0, L/2)
// (both follow from sin(theta) = (e^{i theta} - e^{-i theta})/2i; no prefix scan, so the FP32
// error is that of the FFT).
//
// Depth layout: the index n is split by residue mod R = 2 NCTA, n = r + R m, m in [0, M),
// M = L/R.  CTA j holds the two residue rows {j, R - j} (CTA 0: {0, R/2}).  The mirror
// L - n of a row-r point lies in row R - r, so the pre-processing above is local.
// FFT_L = local M-point FFTs of every residue row (4 per CTA: two rows, u and v), the twiddle
// w_L^{r k1}, then for every k1 an R-point DFT across the residues:
//   X[k1 + M k2] = sum_r w_R^{r k2} (w_L^{r k1} FFT_M(row r)[k1]).
// CTA j owns k1 in [jQ, (j+1)Q), Q = M/NCTA: the twiddled FFT outputs reach the CTA owning
// their k1 (the one all-to-all exchange of a transform) either pushed by remote stores before
// the barrier or pulled by remote loads after it (template flag PUSH); the owner keeps the
// outputs k = k1 + M k2 < L/2 (k2 < R/2): spectral layout, thread (k1', e, h) owning
// S_{2(k1 + M k2) + e} for k2 in [h R/4, (h+1) R/4).  The R-point DFT of a thread pair is
// split by residue parity: thread h transforms the R/2 residues of parity h and the pair swaps
// halves by shuffle.
// The inverse transform (spectral -> depth; the DST-I matrix is symmetric) runs the same
// factors transposed and in reverse order, so it maps the spectral layout back to the depth
// layout, again with one exchange.  Each exchange is one cluster barrier: the exchange area is
// double-buffered by the barrier count's parity, so an area is rewritten only after the barrier
// that follows the reads of it.  Every control decision is derived from values that are
// bitwise identical in all CTAs of the cluster (the descriptor, and norm partials summed in
// CTA order), so all CTAs pass the same barriers.
#pragma once
#include <cooperative_groups.h>

#include "march_kernel.cuh"

namespace sssp {

template <int LOG2L, int NCTA, bool PUSH>
struct CCfg {
  static constexpr int L = 1 << LOG2L;
  static constexpr int R = 2 * NCTA;
  static constexpr int LOG2R = NCTA == 8 ? 4 : 5;
  static constexpr int LOG2M = LOG2L - LOG2R;
  static constexpr int M = 1 << LOG2M;
  static constexpr int Q = M / NCTA;
  static constexpr int LOG2Q = LOG2M - (LOG2R - 1);
  static constexpr int NT = 4 * Q;        // threads: (k1', e, h)
  static constexpr int SV = R / 4;        // spectral values per thread
  static constexpr int H = R / 2;         // size of each thread's half DFT
  static constexpr int P4 = 4 * M;        // points of the four local FFTs
  static constexpr int PAD4 = P4 + P4 / 16;
  static constexpr int NW = NT / 32;
  static constexpr int DV = 2 * M / NT;   // depth points per thread in element-wise loops
  // bufA, bufB, E0, E1 (padded) | X, wL rows, c rows (2M each) | twM (M) | wR (H)
  // | part (2 parities x NCTA CTA partials of the stop test) | V rows (2M floats) | red (2 NW)
  static constexpr size_t SMEM =
      sizeof(float2) * (4 * size_t(PAD4) + 6 * M + M + H + 2 * NCTA) + sizeof(float) * (2 * M + 2 * NW);
  static constexpr size_t SMEM_CPLX = SMEM + sizeof(float) * 2 * M;
  static_assert(NCTA == 8 || NCTA == 16, "cluster of 8 or 16 CTAs");
  static_assert(NT >= 32 && NT % 32 == 0 && M >= 64, "grid too small for this cluster");
};

template <int LOG2L, int NCTA, bool PUSH>
struct CSmem {
  float2 *bufA, *bufB, *E[2], *X, *wLs, *cs, *twM, *wR, *part;
  float *Vs, *red, *Vis;
  __device__ __forceinline__ explicit CSmem(unsigned char* base) {
    using C = CCfg<LOG2L, NCTA, PUSH>;
    bufA = reinterpret_cast<float2*>(base);
    bufB = bufA + C::PAD4;
    E[0] = bufB + C::PAD4;
    E[1] = E[0] + C::PAD4;
    X = E[1] + C::PAD4;
    wLs = X + 2 * C::M;
    cs = wLs + 2 * C::M;
    twM = cs + 2 * C::M;
    wR = twM + C::M;
    part = wR + C::H;
    Vs = reinterpret_cast<float*>(part + 2 * NCTA);
    red = Vs + 2 * C::M;
    Vis = red + 2 * C::NW;  // complex-profile kernel only
  }
};

// residue held in row `row` of CTA j, and the (CTA, row) holding residue r
template <int NCTA>
__device__ __forceinline__ int res_of(int j, int row) {
  return row == 0 ? j : (j == 0 ? NCTA : 2 * NCTA - j);
}
template <int NCTA>
__device__ __forceinline__ void owner_of(int r, int& own, int& row) {
  if (r == 0) {
    own = 0;
    row = 0;
  } else if (r == NCTA) {
    own = 0;
    row = 1;
  } else if (r < NCTA) {
    own = r;
    row = 0;
  } else {
    own = 2 * NCTA - r;
    row = 1;
  }
}
// position of the mirror point L - n of (row, m) in CTA j
template <int M>
__device__ __forceinline__ int mirror_pos(int j, int row, int m) {
  if (j == 0) return row == 0 ? ((M - m) & (M - 1)) : (M + M - 1 - m);
  return (1 - row) * M + (M - 1 - m);
}

// One Stockham pass of radix RAD over span NS on the four local M-point FFTs (FFT f owns
// points [f M, (f+1) M) of the batch): ld(f, i) gives input i of FFT f, st(f, o, v) takes
// output o.
template <int LOG2M, int NT, int RAD, int NS, class LD, class ST>
__device__ __forceinline__ void cpass(const LD& ld, const ST& st, const float2* __restrict__ tw) {
  constexpr int M = 1 << LOG2M, NB = M / RAD, PER = 4 * NB / NT;
  static_assert(PER >= 1 && PER * NT == 4 * NB, "butterflies per thread");
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int jb = threadIdx.x + q * NT;
    const int f = jb / NB, jj = jb & (NB - 1);
    float2 v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = ld(f, jj + r * NB);
    const int k = jj & (NS - 1);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[NS - 8 + (r - 1) * NS + k]);
    }
    dftR<RAD>(v);
    const int base = (jj - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) st(f, base + r * NS, v[r]);
  }
}

template <int M>
struct LdBuf {
  const float2* src;
  __device__ __forceinline__ float2 operator()(int f, int i) const { return src[pidx(f * M + i)]; }
};
template <int M>
struct StBuf {
  float2* dst;
  __device__ __forceinline__ void operator()(int f, int o, float2 v) const { dst[pidx(f * M + o)] = v; }
};
// last forward pass: twiddle w_L^{r k1} of the row, pushed into the exchange area of the CTA
// that owns k1, at ((2 r + e) Q + k1 - its first k1)
// (pull: into this CTA's own area at (f M + k1), read by the owner of k1 after the barrier)
template <int LOG2L, int NCTA, bool PUSH>
struct StExch {
  float2* E;  // this CTA's exchange area (mapped to the owner per store when pushing)
  const float2* wLs;
  int j;
  __device__ __forceinline__ void operator()(int f, int o, float2 v) const {
    using C = CCfg<LOG2L, NCTA, PUSH>;
    const float2 w = cmul(v, wLs[(f >> 1) * C::M + o]);
    if constexpr (PUSH) {
      const int r = res_of<NCTA>(j, f >> 1);
      float2* Eo = cooperative_groups::this_cluster().map_shared_rank(E, o >> C::LOG2Q);
      Eo[pidx((2 * r + (f & 1)) * C::Q + (o & (C::Q - 1)))] = w;
    } else {
      E[pidx(f * C::M + o)] = w;
    }
  }
};

// passes of span NS .. M after the first; the last one stores with `last`
template <int LOG2M, int NT, int NS, class STL>
__device__ __forceinline__ void cfft_rest(float2* src, float2* dst, const float2* tw, const STL& last) {
  constexpr int M = 1 << LOG2M;
  constexpr int RAD = (M / NS) >= 8 ? 8 : (M / NS);
  if constexpr (NS * RAD == M) {
    cpass<LOG2M, NT, RAD, NS>(LdBuf<M>{src}, last, tw);
  } else {
    cpass<LOG2M, NT, RAD, NS>(LdBuf<M>{src}, StBuf<M>{dst}, tw);
    __syncthreads();
    cfft_rest<LOG2M, NT, NS * RAD>(dst, src, tw, last);
  }
}
// number of passes of an M-point FFT (first radix-8 pass included); passes alternate writing
// A, B, A, ... starting with A, so the last one writes A when their number is odd
template <int LOG2M>
struct CPasses {
  static constexpr int NP = (LOG2M + 2) / 3;
  static constexpr bool LAST_IN_A = (NP % 2) == 1;
};

__device__ __forceinline__ float2 mul_ihalf(float2 x) { return make_float2(-0.5f * x.y, 0.5f * x.x); }

// Forward pre-processing loader (first pass): u or v of the depth values X (times V when
// WITHV) for FFT f = 2 row + e.
template <int LOG2L, int NCTA, bool PUSH, bool WITHV, bool CPLX>
struct LdPre {
  const float2* X;
  const float* Vs;
  const float* Vis;
  const float2* cs;
  int j;
  __device__ __forceinline__ float2 val(int p) const {
    const float2 x = X[p];
    if constexpr (!WITHV) return x;
    else if constexpr (CPLX) return cmul(make_float2(Vs[p], Vis[p]), x);
    else return Vs[p] * x;
  }
  __device__ __forceinline__ float2 operator()(int f, int m) const {
    constexpr int M = CCfg<LOG2L, NCTA, PUSH>::M;
    const int row = f >> 1;
    const int p = row * M + m;
    const float2 x = val(p), xm = val(mirror_pos<M>(j, row, m));
    return (f & 1) ? cmul(x + xm, cs[p]) : x - xm;
  }
};

// Inverse first pass: the values the other CTAs pushed for residue row f >> 1, term f & 1, at
// (f M + k1) of this CTA's exchange area, times w_L^{r k1}.
// (pull: read from the area of the CTA owning k1, at ((2 r + e) Q + k1 - its first k1))
template <int LOG2L, int NCTA, bool PUSH>
struct LdExch {
  const float2* E;
  const float2* wLs;
  int j;
  __device__ __forceinline__ float2 operator()(int f, int k1) const {
    using C = CCfg<LOG2L, NCTA, PUSH>;
    float2 z;
    if constexpr (PUSH) {
      z = E[pidx(f * C::M + k1)];
    } else {
      const int r = res_of<NCTA>(j, f >> 1);
      const float2* Eo = cooperative_groups::this_cluster().map_shared_rank(E, k1 >> C::LOG2Q);
      z = Eo[pidx((2 * r + (f & 1)) * C::Q + (k1 & (C::Q - 1)))];
    }
    return cmul(z, wLs[(f >> 1) * C::M + k1]);
  }
};

// thread's spectral coordinates
template <int LOG2L, int NCTA, bool PUSH>
struct Spec {
  int h, e, k1;  // k1: global
  __device__ __forceinline__ Spec(int j) {
    using C = CCfg<LOG2L, NCTA, PUSH>;
    const int t = threadIdx.x;
    h = t & 1;
    e = (t >> 1) & 1;
    k1 = j * C::Q + (t >> 2);
  }
  __device__ __forceinline__ int mode(int s) const {
    using C = CCfg<LOG2L, NCTA, PUSH>;
    return 2 * (k1 + C::M * (h * C::SV + s)) + e;
  }
};

// Forward DST-I of the depth values in X (times V when WITHV): out[s] = S at sp.mode(s).
// Uses bufA, bufB and the exchange area of parity ph (one cluster barrier; ph advances).
template <int LOG2L, int NCTA, bool PUSH, bool WITHV, bool CPLX>
__device__ __forceinline__ void cdst_fwd(CSmem<LOG2L, NCTA, PUSH>& sm, int j, const Spec<LOG2L, NCTA, PUSH>& sp, int& ph,
                                         float2 (&out)[CCfg<LOG2L, NCTA, PUSH>::SV]) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  constexpr int M = C::M;
  float2* E = sm.E[ph & 1];
  cpass<C::LOG2M, C::NT, 8, 1>(LdPre<LOG2L, NCTA, PUSH, WITHV, CPLX>{sm.X, sm.Vs, sm.Vis, sm.cs, j}, StBuf<M>{sm.bufA},
                              sm.twM);
  __syncthreads();
  cfft_rest<C::LOG2M, C::NT, 8>(sm.bufA, sm.bufB, sm.twM, StExch<LOG2L, NCTA, PUSH>{E, sm.wLs, j});
  cooperative_groups::this_cluster().sync();  // the pushed values are visible after it
  ++ph;
  // R-point DFT across residues, split by residue parity over the thread pair (h = 0, 1)
  float2 D[C::H];
  const int k1l = sp.k1 & (C::Q - 1);
#pragma unroll
  for (int s = 0; s < C::H; ++s) {
    if constexpr (PUSH) {
      D[s] = E[pidx((2 * (2 * s + sp.h) + sp.e) * C::Q + k1l)];
    } else {
      int own, row;
      owner_of<NCTA>(2 * s + sp.h, own, row);
      D[s] = cooperative_groups::this_cluster().map_shared_rank(E, own)[pidx((2 * row + sp.e) * M + sp.k1)];
    }
  }
  dftN<C::H>(D);
  if (sp.h) {
#pragma unroll
    for (int s = 1; s < C::H; ++s) D[s] = cmul(D[s], sm.wR[s]);
  }
#pragma unroll
  for (int s = 0; s < C::SV; ++s) {
    const float2 send = sp.h ? D[s] : D[C::SV + s];
    const float2 mine = sp.h ? D[C::SV + s] : D[s];
    const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1), __shfl_xor_sync(0xffffffffu, send.y, 1));
    out[s] = mul_ihalf(mine + recv);
  }
}

// Where the inverse transform's depth values go.
constexpr int kSinkX = 0;      // shared X (for the next forward transform)
constexpr int kSinkTL = 1;     // a TL row in global memory
constexpr int kSinkField = 2;  // the physical envelope in global memory

// First half of the inverse DST-I: from the spectral values in[s] (at sp.mode(s)), the
// transposed R-point DFTs into the exchange area of parity ph; then the cluster barrier.
template <int LOG2L, int NCTA, bool PUSH>
__device__ __forceinline__ void cdst_inv_begin(CSmem<LOG2L, NCTA, PUSH>& sm, const Spec<LOG2L, NCTA, PUSH>& sp, int& ph,
                                               const float2 (&in)[CCfg<LOG2L, NCTA, PUSH>::SV]) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  float2* E = sm.E[ph & 1];
  float2 W[C::H];
#pragma unroll
  for (int s = 0; s < C::SV; ++s) {
    const float2 u = mul_ihalf(in[s]);
    const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, u.x, 1), __shfl_xor_sync(0xffffffffu, u.y, 1));
    W[s] = sp.h ? o : u;
    W[C::SV + s] = sp.h ? u : o;
  }
  if (sp.h) {
#pragma unroll
    for (int s = 1; s < C::H; ++s) W[s] = cmul(W[s], sm.wR[s]);
  }
  dftN<C::H>(W);
  // push Z_r[k1] to the CTA holding residue r, at ((2 row + e) M + k1); or keep it here at
  // ((2 r + e) Q + k1') for that CTA to pull
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int k1l = sp.k1 & (C::Q - 1);
#pragma unroll
  for (int s = 0; s < C::H; ++s) {
    if constexpr (PUSH) {
      int own, row;
      owner_of<NCTA>(2 * s + sp.h, own, row);
      cl.map_shared_rank(E, own)[pidx((2 * row + sp.e) * C::M + sp.k1)] = W[s];
    } else {
      E[pidx((2 * (2 * s + sp.h) + sp.e) * C::Q + k1l)] = W[s];
    }
  }
  cl.sync();
  ++ph;
}

// Second half: gather this CTA's residue rows from the exchange area written before the last
// barrier (parity ph - 1), local FFTs, transposed pre-processing into the sink.
template <int LOG2L, int NCTA, bool PUSH, int SINK>
__device__ __forceinline__ void cdst_inv_end(CSmem<LOG2L, NCTA, PUSH>& sm, int j, int ph, float2* fout, float* tlrow,
                                             float lr) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  constexpr int M = C::M;
  cpass<C::LOG2M, C::NT, 8, 1>(LdExch<LOG2L, NCTA, PUSH>{sm.E[(ph - 1) & 1], sm.wLs, j}, StBuf<M>{sm.bufA}, sm.twM);
  __syncthreads();
  constexpr bool inA = CPasses<C::LOG2M>::LAST_IN_A;
  float2* F = inA ? sm.bufA : sm.bufB;
  cfft_rest<C::LOG2M, C::NT, 8>(sm.bufA, sm.bufB, sm.twM, StBuf<M>{F});
  __syncthreads();
  // x_n = u'_n - u'_{L-n} + c_n v'_n + c_{L-n} v'_{L-n}
#pragma unroll
  for (int q = 0; q < C::DV; ++q) {
    const int i = threadIdx.x + q * C::NT;
    const int row = i >> C::LOG2M, m = i & (M - 1);
    const int mp = mirror_pos<M>(j, row, m);
    const int mrow = mp >> C::LOG2M, mm = mp & (M - 1);
    const float2 xu = F[pidx(2 * row * M + m)], xum = F[pidx(2 * mrow * M + mm)];
    const float2 xv = F[pidx((2 * row + 1) * M + m)], xvm = F[pidx((2 * mrow + 1) * M + mm)];
    float2 x = (xu - xum) + cmul(sm.cs[i], xv) + cmul(sm.cs[mp], xvm);
    const int n = res_of<NCTA>(j, row) + C::R * m;
    if (n == 0) x = make_float2(0.f, 0.f);
    if constexpr (SINK == kSinkX) {
      sm.X[i] = x;
    } else if constexpr (SINK == kSinkField) {
      fout[n] = x;
    } else {
      if (n >= 1) tlrow[n - 1] = fmaf(-10.f, log10f(cabs2(x)), lr);
    }
  }
  if constexpr (SINK == kSinkX) __syncthreads();
}

template <int LOG2L, int NCTA, bool PUSH>
__device__ __forceinline__ void cload_tables(CSmem<LOG2L, NCTA, PUSH>& sm, int j, const float2* __restrict__ twM_g,
                                             const float2* __restrict__ wL_g, const float2* __restrict__ c_g,
                                             const float2* __restrict__ wR_g) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  for (int i = threadIdx.x; i < 2 * C::M; i += C::NT) {
    const int row = i >> C::LOG2M, m = i & (C::M - 1);
    const int r = res_of<NCTA>(j, row);
    sm.wLs[i] = wL_g[r * C::M + m];
    sm.cs[i] = c_g[r * C::M + m];
  }
  for (int i = threadIdx.x; i < C::M; i += C::NT) sm.twM[i] = twM_g[i];
  for (int i = threadIdx.x; i < C::H; i += C::NT) sm.wR[i] = wR_g[i];
}

template <int LOG2L, int NCTA, bool PUSH, bool CPLX>
__device__ __forceinline__ void cload_V(CSmem<LOG2L, NCTA, PUSH>& sm, int j, const SolveDesc& d, int node) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  const float* Vg = d.V + (size_t)node * C::L;
  const float* Vig = CPLX ? d.Vi + (size_t)node * C::L : nullptr;
  for (int i = threadIdx.x; i < 2 * C::M; i += C::NT) {
    const int row = i >> C::LOG2M, m = i & (C::M - 1);
    const int n = res_of<NCTA>(j, row) + C::R * m;
    sm.Vs[i] = Vg[n];
    if constexpr (CPLX) sm.Vis[i] = Vig[n];
  }
}

// ---------------------------------------------------------------------------------------
// The persistent cluster march: cluster blockIdx.x / NCTA marches solve descs[that].
// ---------------------------------------------------------------------------------------
template <int LOG2L, int NCTA, bool PUSH, bool CPLX>
__global__ void __launch_bounds__(CCfg<LOG2L, NCTA, PUSH>::NT, 1)
    sssp_march_cluster_kernel(const SolveDesc* __restrict__ descs, const float2* __restrict__ twM_g,
                              const float2* __restrict__ wL_g, const float2* __restrict__ c_g,
                              const float2* __restrict__ wR_g) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  constexpr int SV = C::SV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CSmem<LOG2L, NCTA, PUSH> sm(smem_raw);
  __shared__ SolveDesc d;
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int j = int(cl.block_rank());
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  {
    const int* src = reinterpret_cast<const int*>(descs + blockIdx.x / NCTA);
    int* dst = reinterpret_cast<int*>(&d);
    for (int i = t; i < int(sizeof(SolveDesc) / sizeof(int)); i += C::NT) dst[i] = src[i];
  }
  cload_tables<LOG2L, NCTA, PUSH>(sm, j, twM_g, wL_g, c_g, wR_g);
  __syncthreads();
  const Spec<LOG2L, NCTA, PUSH> sp(j);
  float2 y[SV];
#pragma unroll
  for (int s = 0; s < SV; ++s) y[s] = d.yhat[sp.mode(s)];
  const float out_scale = 2.0f / float(C::L);
  const bool iso = d.terms <= 1;
  const float tol2f = float(d.tol2);  // the FP32 prefilter of the FP64 stop test
  int status = kStatusOk;
  unsigned int ndst = 0;
  int nrec = 0;
  int ph = 0;
  int node = d.node0;
  double next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
  if (!iso) cload_V<LOG2L, NCTA, PUSH, CPLX>(sm, j, d, node);
  __syncthreads();

  auto record = [&](int s) {
    float2 o[SV];
#pragma unroll
    for (int i = 0; i < SV; ++i) o[i] = out_scale * y[i];
    cdst_inv_begin<LOG2L, NCTA, PUSH>(sm, sp, ph, o);
    const float lr = float(10.0 * log10(d.r0 + double(s + 1) * d.dr));
    cdst_inv_end<LOG2L, NCTA, PUSH, kSinkTL>(sm, j, ph, nullptr, d.tl + (size_t)(d.rec0 + nrec) * d.N, lr);
    ++ndst;
    ++nrec;
  };

  if (iso) {
    float4 G[SV];
#pragma unroll
    for (int s = 0; s < SV; ++s) G[s] = d.G[sp.mode(s)];
    for (int s = 0; s < d.steps; ++s) {
#pragma unroll
      for (int i = 0; i < SV; ++i) y[i] = ffmul(G[i], y[i]);
      const long long gs = d.step0 + s + 1;
      if (d.tl_every > 0 && gs % d.tl_every == 0) record(s);
    }
  } else {
    for (int s = 0; s < d.steps && status == kStatusOk; ++s) {
      const double rmid = d.r0 + (double(s) + 0.5) * d.dr;
      if (rmid >= next_r) {
        while (node + 1 < d.nodes && d.node_r[node + 1] <= rmid) ++node;
        next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
        cload_V<LOG2L, NCTA, PUSH, CPLX>(sm, j, d, node);  // read after the barriers of the stage's first transform
      }
      for (int jj = 0; jj < d.p && status == kStatusOk; ++jj) {
        float2 acc[SV], tp[SV], t0[SV], Bj[SV];
#pragma unroll
        for (int i = 0; i < SV; ++i) {
          const int md = sp.mode(i);
          Bj[i] = d.B[(size_t)jj * C::L + md];
          t0[i] = cmul(d.A[(size_t)jj * C::L + md], y[i]);
          acc[i] = make_float2(0.f, 0.f);
        }
        cdst_inv_begin<LOG2L, NCTA, PUSH>(sm, sp, ph, t0);
        cdst_inv_end<LOG2L, NCTA, PUSH, kSinkX>(sm, j, ph, nullptr, nullptr, 0.f);  // t_0 in depth space
        ++ndst;
        float first = 0.f;
        for (int m = 1; m < d.terms; ++m) {
          cdst_fwd<LOG2L, NCTA, PUSH, true, CPLX>(sm, j, sp, ph, tp);  // T(V t_{m-1})
          ++ndst;
          float nt = 0.f, nw = 0.f;
#pragma unroll
          for (int i = 0; i < SV; ++i) {
            tp[i] = cmul(Bj[i], tp[i]);
            acc[i] = acc[i] + tp[i];
            nt += cabs2(tp[i]);
            nw += cabs2(t0[i] + acc[i]);
          }
          if (m == d.terms - 1) break;
          // CTA partials: warp butterflies, then warps in order by thread 0, published for
          // the other CTAs in the part slot of this exchange's parity
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            nt += __shfl_xor_sync(0xffffffffu, nt, o);
            nw += __shfl_xor_sync(0xffffffffu, nw, o);
          }
          if (lane == 0) {
            sm.red[2 * warp] = nt;
            sm.red[2 * warp + 1] = nw;
          }
          __syncthreads();
          const int pbase = (ph & 1) * NCTA;
          if (warp == 0) {  // the CTA total, pushed by lane c into slot j of CTA c
            float a = 0.f, b = 0.f;
            for (int w = 0; w < C::NW; ++w) {
              a += sm.red[2 * w];
              b += sm.red[2 * w + 1];
            }
            if (lane < NCTA) cl.map_shared_rank(sm.part, lane)[pbase + j] = make_float2(a, b);
          }
          cdst_inv_begin<LOG2L, NCTA, PUSH>(sm, sp, ph, tp);  // (its cluster barrier publishes part)
          float snt = 0.f, snw = 0.f;
          for (int c = 0; c < NCTA; ++c) {
            const float2 pc = sm.part[pbase + c];
            snt += pc.x;
            snw += pc.y;
          }
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
          cdst_inv_end<LOG2L, NCTA, PUSH, kSinkX>(sm, j, ph, nullptr, nullptr, 0.f);  // t_m in depth space
          ++ndst;
        }
        const float2 bj = d.beta[jj];
#pragma unroll
        for (int i = 0; i < SV; ++i) {
          const float4 rj = d.R[(size_t)jj * C::L + sp.mode(i)];
          y[i] = ffmul(rj, y[i]) + cmul(bj, acc[i]);
        }
      }
      if (status != kStatusOk) break;
      const long long gs = d.step0 + s + 1;
      if (d.tl_every > 0 && gs % d.tl_every == 0) record(s);
    }
  }
#pragma unroll
  for (int s = 0; s < SV; ++s) d.yhat[sp.mode(s)] = y[s];
  {
    float2 o[SV];
#pragma unroll
    for (int i = 0; i < SV; ++i) o[i] = out_scale * y[i];
    cdst_inv_begin<LOG2L, NCTA, PUSH>(sm, sp, ph, o);
    cdst_inv_end<LOG2L, NCTA, PUSH, kSinkField>(sm, j, ph, d.field, nullptr, 0.f);
    ++ndst;
  }
  if (t == 0 && j == 0) {
    if (status != kStatusOk) atomicMax(d.status, status);
    atomicAdd(d.ndst, (unsigned long long)ndst);
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// DST-I of one field per cluster: out = scale * DST(in); field b = blockIdx.x / NCTA reads N
// values at in + b * in_stride (n = 1..N) and writes L values at out + b * out_stride.
template <int LOG2L, int NCTA, bool PUSH>
__global__ void __launch_bounds__(CCfg<LOG2L, NCTA, PUSH>::NT, 1)
    sssp_dst_cluster_kernel(const float2* __restrict__ in, float2* __restrict__ out, float scale,
                            const float2* __restrict__ twM_g, const float2* __restrict__ wL_g,
                            const float2* __restrict__ c_g, const float2* __restrict__ wR_g, long long in_stride,
                            long long out_stride) {
  using C = CCfg<LOG2L, NCTA, PUSH>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CSmem<LOG2L, NCTA, PUSH> sm(smem_raw);
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int j = int(cl.block_rank());
  const long long b = blockIdx.x / NCTA;
  in += b * in_stride;
  out += b * out_stride;
  cload_tables<LOG2L, NCTA, PUSH>(sm, j, twM_g, wL_g, c_g, wR_g);
  for (int i = threadIdx.x; i < 2 * C::M; i += C::NT) {
    const int row = i >> C::LOG2M, m = i & (C::M - 1);
    const int n = res_of<NCTA>(j, row) + C::R * m;
    sm.X[i] = (n == 0) ? make_float2(0.f, 0.f) : in[n - 1];
  }
  __syncthreads();
  const Spec<LOG2L, NCTA, PUSH> sp(j);
  int ph = 0;
  float2 o[C::SV];
  cdst_fwd<LOG2L, NCTA, PUSH, false, false>(sm, j, sp, ph, o);
#pragma unroll
  for (int s = 0; s < C::SV; ++s) {
    const int md = sp.mode(s);
    out[md] = (md == 0) ? make_float2(0.f, 0.f) : scale * o[s];  // S_0 = 0 exactly
  }
  cl.sync();
}

}  // namespace sssp
