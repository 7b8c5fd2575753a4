// Batched march with the DST-I as a dense GEMM on the tensor cores (a precision variant).
//
// For a batch of B solves of one grid size (L = N + 1 a power of two, L >= 128), every
// transform of the march is applied to all B fields at once as Y = S X with
// S[m][n] = sin(pi n m/L) (L x L with the zero row and column m = 0 / n = 0 of the index
// convention of the FFT marcher, real, symmetric) and X the L x C real matrix of the fields'
// components, column 2b the real and 2b + 1 the imaginary part of field b (C = 2B rounded up to
// the tile width, extra columns zero).  The contraction is this file's own kernel:
//   PE_GEMM_BF16X3  S = S_hi + S_lo, X = X_hi + X_lo with BF16 parts, three tcgen05.mma
//                   products (hi hi + hi lo + lo hi) into one FP32 accumulator in tensor memory;
//   PE_GEMM_TF32    one tcgen05.mma kind::tf32 product of the TF32-rounded operands;
//   PE_GEMM_3XTF32  the hi/lo split with TF32 parts, three kind::tf32 products;
//   PE_GEMM_FP32    a CUDA-core FP32 GEMM (the reference the others are measured against).
// A cluster of kKS CTAs owns a 128 x 32 kKS output tile, each CTA one K range of it: one thread
// issues TMA loads of 128-byte swizzled K slices of S and X (the hi and lo planes of a split
// operand in one 3D load) into a multi-stage shared-memory ring, another issues the MMAs
// (K-major operands, the accumulator in tensor memory), then the partial tiles are summed over
// the cluster's distributed shared memory and each CTA runs the step's element-wise work for
// its share of the rows in the epilogue (its operand loads issued before the main loop),
// writing the next GEMM's operand (already split) directly:
//   after a transform to depth space:    X' = V .* Y                 (the Neumann term's V t)
//   after a transform to spectral space: t_m = B_j .* Y, acc += t_m, X' = t_m.
// So one Neumann term is two GEMM launches and nothing else; the stage start (t_0 = A_j y) and
// end (y = R_j y + beta_j acc, hi/lo multiplier) are small element-wise kernels.  The tables and
// the arithmetic are the FFT marcher's.  The series takes a fixed number of terms (the plans'
// neumann_terms) for every solve, so the batch stays in lockstep; one range step is captured in
// a CUDA graph and replayed.
//
// The dense transform costs 2 L^2 flop per real column against ~5 L log2 L for the FFT, so this
// form is measured for its accuracy per precision and for the tensor pipe, not offered as the
// fast path.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sssp.h"
#include "plan_internal.h"
#include "umma.cuh"

namespace {

constexpr int kBM = 128;        // output rows per tile (modes or depths): the MMA's M, one TMEM lane each
constexpr int kKS = 2;          // K splits per output tile = CTAs per cluster (1, 2 or 4)
constexpr int kBN = 32 * kKS;   // output columns per tile: the MMA's N, as many TMEM columns
constexpr int kRowBytes = 128;  // one swizzled K slice row: 64 BF16 or 32 FP32 values
constexpr int kThreads = 128;
constexpr uint64_t kWaitNs = 500000000ull;  // every barrier wait gives up after 0.5 s
constexpr int kStatusTimeout = 5;

enum Epi { kEpiTimesV = 0, kEpiTerm = 1, kEpiTermLast = 2, kEpiOut = 3 };

struct GemmSolve {  // per-solve tables (device, L-indexed, index 0 the zero pad)
  const float2* A;
  const float2* B;
  const float4* R;
  const float* V;
  float2 beta[sssp::kMaxStages];
};

struct EpiArgs {
  const GemmSolve* solves;
  float2* ACC;   // B x L Neumann sums (spectral)
  void* Xhi;     // next GEMM operand, C x L (BF16 for BF16X3, FP32 otherwise)
  void* Xlo;     // its low part (split modes)
  float* Gout;   // C x L FP32 output (read-out)
  int* status;   // error word: a barrier wait that ran out
  int L, B, j;
};

__device__ __forceinline__ float tf32_round(float x) {
  // to the nearest value with a 10-bit mantissa (TF32), ties away from zero
  unsigned u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// X operand element (column col, row m) in the mode's representation
template <int MODE>
__device__ __forceinline__ void put_x(void* hi, void* lo, size_t idx, float v) {
  if constexpr (MODE == PE_GEMM_BF16X3) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(hi)[idx] = h;
    static_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
  } else if constexpr (MODE == PE_GEMM_3XTF32) {
    const float h = tf32_round(v);
    static_cast<float*>(hi)[idx] = h;
    static_cast<float*>(lo)[idx] = v - h;
  } else if constexpr (MODE == PE_GEMM_TF32) {
    static_cast<float*>(hi)[idx] = tf32_round(v);
  } else {
    static_cast<float*>(hi)[idx] = v;
  }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// the epilogue of one output pair (row m; columns col = 2b and 2b + 1 of field b)
template <int MODE, int EPI>
__device__ __forceinline__ void epi_pair(const EpiArgs& a, int m, int col, float re, float im) {
  const int b = col >> 1;
  if (b >= a.B) return;  // padding columns stay zero
  const size_t L = size_t(a.L), ir = size_t(col) * L + m, ii = ir + L;
  if constexpr (EPI == kEpiOut) {
    a.Gout[ir] = re;
    a.Gout[ii] = im;
  } else if constexpr (EPI == kEpiTimesV) {
    const float v = a.solves[b].V[m];
    put_x<MODE>(a.Xhi, a.Xlo, ir, v * re);
    put_x<MODE>(a.Xhi, a.Xlo, ii, v * im);
  } else {
    const float2 t = cmulf(a.solves[b].B[size_t(a.j) * L + m], make_float2(re, im));
    float2* acc = a.ACC + size_t(b) * L + m;
    const float2 s = *acc;
    *acc = make_float2(s.x + t.x, s.y + t.y);
    if constexpr (EPI == kEpiTerm) {
      put_x<MODE>(a.Xhi, a.Xlo, ir, t.x);
      put_x<MODE>(a.Xhi, a.Xlo, ii, t.y);
    }
  }
}

template <typename T>
__device__ __forceinline__ T* ldg_ptr(T* const* p) {  // a pointer field of a read-only table
  return reinterpret_cast<T*>(__ldg(reinterpret_cast<const unsigned long long*>(p)));
}

// The epilogue of 16 output pairs (row m; fields b0 .. b0 + 15, columns 2b and 2b + 1), the
// same arithmetic as epi_pair in two parts: load() issues every operand load of the 16 pairs
// (the kernel calls it before its main loop, so the loads complete under the contraction) and
// apply() takes the accumulator values and does the stores.
template <int MODE, int EPI>
struct EpiOps {
  float vv[16];
  float2 bb[16], ac[16];
  __device__ __forceinline__ void load(const EpiArgs& a, int m, int col0) {
    const int b0 = col0 >> 1;
    const size_t L = size_t(a.L);
    if constexpr (EPI == kEpiTimesV) {
      const float* vp[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) vp[i] = (b0 + i < a.B) ? ldg_ptr(&a.solves[b0 + i].V) : nullptr;
#pragma unroll
      for (int i = 0; i < 16; ++i) vv[i] = vp[i] ? __ldg(vp[i] + m) : 0.f;
    } else if constexpr (EPI == kEpiTerm || EPI == kEpiTermLast) {
      const float2* bp[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) bp[i] = (b0 + i < a.B) ? ldg_ptr(&a.solves[b0 + i].B) : nullptr;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        bb[i] = bp[i] ? __ldg(bp[i] + size_t(a.j) * L + m) : make_float2(0.f, 0.f);
        ac[i] = bp[i] ? a.ACC[size_t(b0 + i) * L + m] : make_float2(0.f, 0.f);
      }
    }
  }
  __device__ __forceinline__ void apply(const EpiArgs& a, int m, int col0, const float (&v)[32]) const {
    const int b0 = col0 >> 1;
    const size_t L = size_t(a.L);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (b0 + i >= a.B) continue;  // padding columns stay zero
      const size_t ir = size_t(col0 + 2 * i) * L + m;
      if constexpr (EPI == kEpiOut) {
        a.Gout[ir] = v[2 * i];
        a.Gout[ir + L] = v[2 * i + 1];
      } else if constexpr (EPI == kEpiTimesV) {
        put_x<MODE>(a.Xhi, a.Xlo, ir, vv[i] * v[2 * i]);
        put_x<MODE>(a.Xhi, a.Xlo, ir + L, vv[i] * v[2 * i + 1]);
      } else {
        const float2 t = cmulf(bb[i], make_float2(v[2 * i], v[2 * i + 1]));
        a.ACC[size_t(b0 + i) * L + m] = make_float2(ac[i].x + t.x, ac[i].y + t.y);
        if constexpr (EPI == kEpiTerm) {
          put_x<MODE>(a.Xhi, a.Xlo, ir, t.x);
          put_x<MODE>(a.Xhi, a.Xlo, ir + L, t.y);
        }
      }
    }
  }
};

template <int MODE>
struct Traits {
  static constexpr bool SPLIT = MODE != PE_GEMM_TF32;  // hi/lo operands, three products
  static constexpr bool BF16 = MODE == PE_GEMM_BF16X3;
  static constexpr int EL = BF16 ? 2 : 4;              // operand bytes
  static constexpr int BK = kRowBytes / EL;            // K values per pipeline stage
  static constexpr int A_BYTES = kBM * kRowBytes;      // one S slice (128 rows x 128 B)
  static constexpr int B_BYTES = kBN * kRowBytes;      // one X slice (kBN columns x 128 B)
  // a stage: [S_hi | S_lo | X_hi | X_lo] (split modes: one 3D load each for S and X), or [S | X]
  static constexpr int STAGE_BYTES = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
  static constexpr int STAGES0 = 196608 / STAGE_BYTES;  // ring stages within 192 KB, 2 .. 6
  static constexpr int STAGES = STAGES0 < 2 ? 2 : (STAGES0 > 6 ? 6 : STAGES0);
  static constexpr int P_BYTES = kKS > 1 ? kBN * kBM * 4 : 0;  // FP32 partial tile (reuses the ring)
  static constexpr size_t RING = size_t(STAGES) * STAGE_BYTES;
  static constexpr size_t SMEM = (RING > size_t(P_BYTES) ? RING : size_t(P_BYTES)) + 1024;  // + alignment slack
  static constexpr uint32_t IDESC = umma::instr_desc(kBM, kBN, BF16 ? umma::kFmtBF16 : umma::kFmtTF32);
};

// Y = S X for one 128 x kBN output tile with the fused epilogue (see the file comment), its K
// range split over the kKS CTAs of a thread-block cluster: each CTA contracts L / kKS of K into
// its tensor memory, stores the FP32 partial tile in its shared memory, and after a cluster
// barrier CTA r sums the 128 / kKS rows [r 128 / kKS, ..) of every CTA's partial (distributed
// shared memory, in CTA order) and runs their epilogue.
template <int MODE, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    sssp_gemm_dst_kernel(const __grid_constant__ CUtensorMap mS, const __grid_constant__ CUtensorMap mX, EpiArgs ea) {
  using T = Traits<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[T::STAGES];
  __shared__ __align__(8) uint64_t empty[T::STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = kKS > 1 ? int(cooperative_groups::this_cluster().block_rank()) : 0;
  const int m0 = blockIdx.x * kBM, c0 = blockIdx.y * kBN;
  const int KB = ea.L / T::BK / kKS, kb0 = rank * KB;  // this CTA's K blocks
  // prologue (overlaps the preceding launch under programmatic dependent launch): barriers,
  // tensor memory, tensor-map prefetch; then wait for the preceding grid's results
  if (threadIdx.x == 0) {
    for (int s = 0; s < T::STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(&done, 1);
    abort_flag = 0;
    umma::fence_barrier_init();
    umma::prefetch_tensormap(&mS);
    umma::prefetch_tensormap(&mX);
  }
  if (warp == 0) {
    umma::tmem_alloc(&tmem_base, kBN);
    umma::tmem_relinquish();
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = tmem_base;
  umma::grid_dep_wait();
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(ea.status) != 0)
    abort_flag = 1;  // an earlier launch of the batch gave up: do nothing more
  __syncthreads();
  // this thread's epilogue: 32 columns of one output row; its operands load under the main loop
  constexpr int RP = kBM / kKS;  // rows per CTA after the reduction
  const int erow = kKS > 1 ? rank * RP + int(threadIdx.x) % RP : int(threadIdx.x);
  const int ecol = kKS > 1 ? c0 + 32 * (int(threadIdx.x) / RP) : c0;
  EpiOps<MODE, EPI> ops;
  if (!abort_flag) ops.load(ea, m0 + erow, ecol);

  if (abort_flag) {
    // nothing to load or multiply
  } else if (warp == 0 && lane == 0) {  // TMA producer
    int issued = 0;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % T::STAGES;
      if (kb >= T::STAGES && !umma::mbar_wait(&empty[s], ((kb / T::STAGES) - 1) & 1, kWaitNs)) {
        abort_flag = 1;
        break;
      }
      uint8_t* st = smem + size_t(s) * T::STAGE_BYTES;
      const int kx = (kb0 + kb) * T::BK;
      umma::mbar_expect_tx(&full[s], T::STAGE_BYTES);
      if constexpr (T::SPLIT) {  // both planes (hi, lo) of each operand in one load
        umma::tma_load_3d(st, &mS, &full[s], kx, m0, 0);
        umma::tma_load_3d(st + 2 * T::A_BYTES, &mX, &full[s], kx, c0, 0);
      } else {
        umma::tma_load_2d(st, &mS, &full[s], kx, m0);
        umma::tma_load_2d(st + T::A_BYTES, &mX, &full[s], kx, c0);
      }
      issued = kb + 1;
    }
    // every load issued has landed before the CTA may leave (bounded)
    for (int kb = (issued > T::STAGES ? issued - T::STAGES : 0); kb < issued; ++kb)
      if (!umma::mbar_wait(&full[kb % T::STAGES], (kb / T::STAGES) & 1, kWaitNs)) abort_flag = 1;
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % T::STAGES;
      if (!umma::mbar_wait(&full[s], (kb / T::STAGES) & 1, kWaitNs)) {
        abort_flag = 1;
        break;
      }
      umma::tc_fence_after();
      const uint8_t* st = smem + size_t(s) * T::STAGE_BYTES;
      const uint64_t ah = umma::desc_sw128(st);
      const uint64_t al = umma::desc_sw128(st + (T::SPLIT ? T::A_BYTES : 0));
      const uint64_t bh = umma::desc_sw128(st + (T::SPLIT ? 2 : 1) * T::A_BYTES);
      const uint64_t bl = umma::desc_sw128(st + (T::SPLIT ? 2 * T::A_BYTES + T::B_BYTES : T::A_BYTES));
#pragma unroll
      for (int kk = 0; kk < kRowBytes / 32; ++kk) {  // MMA K steps of 32 bytes (16 BF16 / 8 TF32)
        const uint64_t o = uint64_t(kk * 32) >> 4;
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        if constexpr (T::BF16) {
          umma::mma_bf16(tmem, ah + o, bh + o, T::IDESC, acc);
          umma::mma_bf16(tmem, ah + o, bl + o, T::IDESC, 1u);
          umma::mma_bf16(tmem, al + o, bh + o, T::IDESC, 1u);
        } else {
          umma::mma_tf32(tmem, ah + o, bh + o, T::IDESC, acc);
          if constexpr (T::SPLIT) {
            umma::mma_tf32(tmem, ah + o, bl + o, T::IDESC, 1u);
            umma::mma_tf32(tmem, al + o, bh + o, T::IDESC, 1u);
          }
        }
      }
      umma::mma_commit(&empty[s]);  // the stage is free once these products have read it
    }
    umma::mma_commit(&done);  // arrives when every product issued has completed
  }
  __syncwarp();
  umma::grid_dep_launch();  // the next launch may start its prologue
  // epilogue: every warp reads its 32 accumulator lanes (rows m0 + 32 w + lane)
  const bool skipped = abort_flag != 0;
  const bool ok = !skipped && umma::mbar_wait(&done, 0, kWaitNs);
  umma::tc_fence_after();
  __syncthreads();  // abort_flag is final; the ring is no longer read or written
  const bool good = ok && !abort_flag;
  float v[32];
  if constexpr (kKS == 1) {
    if (good) {
      umma::tmem_ld32(tmem + (uint32_t(32 * warp) << 16), v);
      ops.apply(ea, m0 + erow, ecol, v);
    }
  } else {
    float* part = reinterpret_cast<float*>(smem);  // [kBN columns][128 rows] FP32
    if (good) {
#pragma unroll 1
      for (int cc = 0; cc < kBN; cc += 32) {
        umma::tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(cc), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) part[(cc + i) * kBM + 32 * warp + lane] = v[i];
      }
    }
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cl.sync();  // every CTA's partial is written (every CTA reaches this barrier)
    if (good) {
      const int colb = ecol - c0;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
#pragma unroll
      for (int c = 0; c < kKS; ++c) {
        const float* pc = cl.map_shared_rank(part, c);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += pc[(colb + i) * kBM + erow];
      }
      ops.apply(ea, m0 + erow, ecol, v);
    }
    cl.sync();  // no CTA leaves while its partial may still be read
  }
  if (!good && threadIdx.x == 0 && !skipped) atomicExch(ea.status, kStatusTimeout);
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, kBN);
}

// FP32 reference contraction on the CUDA cores with the same epilogue: 64 x 32 output tiles,
// 256 threads, each 4 rows x one complex column pair.
template <int EPI>
__global__ void __launch_bounds__(256)
    sssp_gemm_dst_fp32_kernel(const float* __restrict__ S, const float* __restrict__ X, EpiArgs ea) {
  constexpr int TM = 64, TN = 32, TK = 32;
  __shared__ float As[TM][TK + 1];
  __shared__ float Bs[TN][TK + 1];
  const int L = ea.L;
  const int m0 = blockIdx.x * TM, c0 = blockIdx.y * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // column pair tx, rows ty + 16 r
  float acc[4][2] = {};
  for (int k0 = 0; k0 < L; k0 += TK) {
    for (int i = threadIdx.x; i < TM * TK; i += 256) {
      const int r = i / TK, k = i % TK;
      As[r][k] = S[size_t(m0 + r) * L + k0 + k];
    }
    for (int i = threadIdx.x; i < TN * TK; i += 256) {
      const int c = i / TK, k = i % TK;
      Bs[c][k] = X[size_t(c0 + c) * L + k0 + k];
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      const float b0 = Bs[2 * tx][k], b1 = Bs[2 * tx + 1][k];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float a = As[ty + 16 * r][k];
        acc[r][0] = fmaf(a, b0, acc[r][0]);
        acc[r][1] = fmaf(a, b1, acc[r][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) epi_pair<PE_GEMM_FP32, EPI>(ea, m0 + ty + 16 * r, c0 + 2 * tx, acc[r][0], acc[r][1]);
}

// element-wise parts of the step, one thread per (field b, mode m)
struct ElemArgs {
  const GemmSolve* solves;
  float2* Y;    // B x L spectral state
  float2* ACC;  // B x L
  void* Xhi;
  void* Xlo;
  int L, B, j;
  float scale;
};

// stage start: t_0 = A_j y (spectral), acc = 0, X <- t_0
template <int MODE>
__global__ void k_stage_start(ElemArgs a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t L = size_t(a.L);
  if (idx >= L * a.B) return;
  const int m = int(idx % L), b = int(idx / L);
  const float2 t0 = cmulf(a.solves[b].A[size_t(a.j) * L + m], a.Y[idx]);
  a.ACC[idx] = make_float2(0.f, 0.f);
  put_x<MODE>(a.Xhi, a.Xlo, size_t(2 * b) * L + m, t0.x);
  put_x<MODE>(a.Xhi, a.Xlo, size_t(2 * b + 1) * L + m, t0.y);
}

// stage end: y = R_j y (hi/lo multiplier) + beta_j acc
__global__ void k_stage_end(ElemArgs a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t L = size_t(a.L);
  if (idx >= L * a.B) return;
  const int m = int(idx % L), b = int(idx / L);
  const GemmSolve& s = a.solves[b];
  const float4 g = s.R[size_t(a.j) * L + m];
  const float2 y = a.Y[idx], acc = a.ACC[idx], bj = s.beta[a.j];
  const float re_lo = fmaf(g.z, y.x, -g.w * y.y), im_lo = fmaf(g.z, y.y, g.w * y.x);
  const float re = fmaf(g.x, y.x, fmaf(-g.y, y.y, re_lo)), im = fmaf(g.x, y.y, fmaf(g.y, y.x, im_lo));
  a.Y[idx] = make_float2(re + fmaf(bj.x, acc.x, -bj.y * acc.y), im + fmaf(bj.x, acc.y, bj.y * acc.x));
}

// X <- scale y (for the depth-space read-out)
template <int MODE>
__global__ void k_out(ElemArgs a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t L = size_t(a.L);
  if (idx >= L * a.B) return;
  const int m = int(idx % L), b = int(idx / L);
  const float2 y = a.Y[idx];
  put_x<MODE>(a.Xhi, a.Xlo, size_t(2 * b) * L + m, a.scale * y.x);
  put_x<MODE>(a.Xhi, a.Xlo, size_t(2 * b + 1) * L + m, a.scale * y.y);
}

// S in the mode's representation (from the FP32 matrix rounded once from FP64)
__global__ void k_split_s(const float* S, void* hi, void* lo, size_t n, int mode) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  switch (mode) {
    case PE_GEMM_BF16X3: put_x<PE_GEMM_BF16X3>(hi, lo, i, S[i]); break;
    case PE_GEMM_3XTF32: put_x<PE_GEMM_3XTF32>(hi, lo, i, S[i]); break;
    case PE_GEMM_TF32: put_x<PE_GEMM_TF32>(hi, lo, i, S[i]); break;
    default: put_x<PE_GEMM_FP32>(hi, lo, i, S[i]); break;
  }
}

// the plans' spectral states (L-indexed) into Y
__global__ void k_gather(const float2* const* yhats, float2* Y, int L, int B) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(L) * B) return;
  Y[idx] = yhats[idx / L][idx % L];
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of a row-major matrix rows x inner (inner contiguous), tiles of box_rows rows x one
// 128-byte slice, 128-byte swizzle.  planes = 2: the hi and lo parts, plane_bytes apart, as a 3D
// map whose box takes both planes in one load.
bool make_map(CUtensorMap* m, void* base, bool bf16, size_t inner, size_t rows, int box_rows, int planes,
              size_t plane_bytes) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const size_t el = bf16 ? 2 : 4;
  const cuuint64_t dims[3] = {cuuint64_t(inner), cuuint64_t(rows), cuuint64_t(planes)};
  const cuuint64_t strides[2] = {cuuint64_t(inner * el), cuuint64_t(plane_bytes)};
  const cuuint32_t box[3] = {cuuint32_t(kRowBytes / el), cuuint32_t(box_rows), cuuint32_t(planes)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, planes > 1 ? 3 : 2, base,
             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct pe_gemm_batch {
  int N = 0, L = 0, B = 0, C = 0, p = 0, terms = 0, mode = 0;
  std::vector<double> sigma;  // k0 dr of every member (the carrier phase per step)
  long long steps_done = 0;
  cudaStream_t stream = nullptr;
  GemmSolve* dSolves = nullptr;
  void* Shi = nullptr;  // L x L operand (BF16 or FP32); FP32 mode: the FP32 matrix
  void* Slo = nullptr;
  void* Xhi[2] = {nullptr, nullptr};  // ping-pong operands C x L
  void* Xlo[2] = {nullptr, nullptr};
  float2* Y = nullptr;
  float2* ACC = nullptr;
  float* G = nullptr;  // C x L read-out
  int* status = nullptr;
  CUtensorMap mS, mX[2];  // S and the ping-pong X operands (split modes: hi and lo planes)
  cudaGraphExec_t step_graph = nullptr;
  unsigned long long gemms_per_step = 0;
  std::string err;
};

namespace {

pe_status gfail(pe_gemm_batch* g, pe_status s, const std::string& m) {
  if (g) g->err = m;
  return s;
}

EpiArgs epi_args(pe_gemm_batch* g, int j, int out_buf) {
  EpiArgs a;
  a.solves = g->dSolves;
  a.ACC = g->ACC;
  a.Xhi = g->Xhi[out_buf];
  a.Xlo = g->Xlo[out_buf];
  a.Gout = g->G;
  a.status = g->status;
  a.L = g->L;
  a.B = g->B;
  a.j = j;
  return a;
}

template <int MODE, int EPI>
cudaError_t launch_gemm_t(pe_gemm_batch* g, int in_buf, const EpiArgs& a) {
  if constexpr (MODE == PE_GEMM_FP32) {
    const dim3 grid(g->L / 64, g->C / 32);
    sssp_gemm_dst_fp32_kernel<EPI><<<grid, 256, 0, g->stream>>>(static_cast<const float*>(g->Shi),
                                                                static_cast<const float*>(g->Xhi[in_buf]), a);
  } else {
    using T = Traits<MODE>;
    static std::mutex mu;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(sssp_gemm_dst_kernel<MODE, EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(T::SMEM));
        if (e != cudaSuccess) return e;
        attr_dev = dev;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g->L / kBM, g->C / kBN, kKS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = T::SMEM;
    cfg.stream = g->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // overlap with the preceding launch
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;  // the K splits of one tile form a cluster
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = kKS;
    cfg.attrs = attr;
    cfg.numAttrs = kKS > 1 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, sssp_gemm_dst_kernel<MODE, EPI>, g->mS, g->mX[in_buf], a);
  }
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_gemm_m(pe_gemm_batch* g, int epi, int in_buf, const EpiArgs& a) {
  switch (epi) {
    case kEpiTimesV: return launch_gemm_t<MODE, kEpiTimesV>(g, in_buf, a);
    case kEpiTerm: return launch_gemm_t<MODE, kEpiTerm>(g, in_buf, a);
    case kEpiTermLast: return launch_gemm_t<MODE, kEpiTermLast>(g, in_buf, a);
    default: return launch_gemm_t<MODE, kEpiOut>(g, in_buf, a);
  }
}

// one GEMM of the operand in buffer in_buf, epilogue writing buffer 1 - in_buf
cudaError_t launch_gemm(pe_gemm_batch* g, int epi, int in_buf, int j) {
  const EpiArgs a = epi_args(g, j, 1 - in_buf);
  ++g->gemms_per_step;
  switch (g->mode) {
    case PE_GEMM_BF16X3: return launch_gemm_m<PE_GEMM_BF16X3>(g, epi, in_buf, a);
    case PE_GEMM_TF32: return launch_gemm_m<PE_GEMM_TF32>(g, epi, in_buf, a);
    case PE_GEMM_3XTF32: return launch_gemm_m<PE_GEMM_3XTF32>(g, epi, in_buf, a);
    default: return launch_gemm_m<PE_GEMM_FP32>(g, epi, in_buf, a);
  }
}

ElemArgs elem_args(pe_gemm_batch* g, int j, int buf) {
  ElemArgs a;
  a.solves = g->dSolves;
  a.Y = g->Y;
  a.ACC = g->ACC;
  a.Xhi = g->Xhi[buf];
  a.Xlo = g->Xlo[buf];
  a.L = g->L;
  a.B = g->B;
  a.j = j;
  a.scale = 1.f;
  return a;
}

int elem_blocks(const ElemArgs& a) { return int((size_t(a.L) * a.B + 255) / 256); }

void stage_start(pe_gemm_batch* g, const ElemArgs& a) {
  const int bl = elem_blocks(a);
  cudaStream_t st = g->stream;
  switch (g->mode) {
    case PE_GEMM_BF16X3: k_stage_start<PE_GEMM_BF16X3><<<bl, 256, 0, st>>>(a); break;
    case PE_GEMM_TF32: k_stage_start<PE_GEMM_TF32><<<bl, 256, 0, st>>>(a); break;
    case PE_GEMM_3XTF32: k_stage_start<PE_GEMM_3XTF32><<<bl, 256, 0, st>>>(a); break;
    default: k_stage_start<PE_GEMM_FP32><<<bl, 256, 0, st>>>(a); break;
  }
}

void stage_out(pe_gemm_batch* g, const ElemArgs& a) {
  const int bl = elem_blocks(a);
  cudaStream_t st = g->stream;
  switch (g->mode) {
    case PE_GEMM_BF16X3: k_out<PE_GEMM_BF16X3><<<bl, 256, 0, st>>>(a); break;
    case PE_GEMM_TF32: k_out<PE_GEMM_TF32><<<bl, 256, 0, st>>>(a); break;
    case PE_GEMM_3XTF32: k_out<PE_GEMM_3XTF32><<<bl, 256, 0, st>>>(a); break;
    default: k_out<PE_GEMM_FP32><<<bl, 256, 0, st>>>(a); break;
  }
}

// enqueue one range step (all stages, the fixed term count) on g->stream:
//   t_0 = A_j y -> X0;  GEMM X0 (depth t_0) epilogue V.*  -> X1
//   m = 1 .. terms-1:   GEMM X1 (spectral)  epilogue t_m = B_j.*, acc += t_m -> X0
//                       GEMM X0 (depth t_m) epilogue V.*  -> X1        (not after the last term)
//   y = R_j y + beta_j acc
pe_status enqueue_step(pe_gemm_batch* g) {
  g->gemms_per_step = 0;
  for (int j = 0; j < g->p; ++j) {
    stage_start(g, elem_args(g, j, 0));
    cudaError_t e = launch_gemm(g, kEpiTimesV, 0, j);
    for (int m = 1; m < g->terms && e == cudaSuccess; ++m) {
      const bool last = (m == g->terms - 1);
      e = launch_gemm(g, last ? kEpiTermLast : kEpiTerm, 1, j);
      if (!last && e == cudaSuccess) e = launch_gemm(g, kEpiTimesV, 0, j);
    }
    if (e != cudaSuccess) return gfail(g, PE_ERR_CUDA, std::string("GEMM launch: ") + cudaGetErrorString(e));
    const ElemArgs ea = elem_args(g, j, 0);
    k_stage_end<<<elem_blocks(ea), 256, 0, g->stream>>>(ea);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(g, PE_ERR_CUDA, cudaGetErrorString(e));
  return PE_OK;
}

}  // namespace

extern "C" {

pe_status pe_gemm_batch_create(pe_gemm_batch** out, pe_plan** plans, int count, int mode) {
  if (!out || !plans || count < 1 || mode < PE_GEMM_FP32 || mode > PE_GEMM_BF16X3) return PE_ERR_ARG;
  *out = nullptr;
  pe_plan* p0 = plans[0];
  if (!p0) return PE_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    pe_plan* p = plans[i];
    if (!p || p->N != p0->N || p->p != p0->p || p->terms != p0->terms || p->dr != p0->dr) {
      p0->err = "GEMM batch: plans must share N, Pade order, term count and dr";
      return PE_ERR_ARG;
    }
    if (!p->field_set || p->terms < 2 || p->nodes != 1 || p->complex_profile || p->bc != PE_BC_DIRICHLET) {
      p0->err = "GEMM batch: every plan needs a field, one real profile node and neumann_terms >= 2";
      return PE_ERR_STATE;
    }
  }
  if (p0->L < kBM || p0->L > 16384 || p0->L / 64 < kKS) {  // every K split gets a whole K block
    p0->err = "GEMM batch: N + 1 must be a power of two in [128, 16384]";
    return PE_ERR_ARG;
  }
  pe_gemm_batch* g = new pe_gemm_batch();
  g->N = p0->N;
  g->L = p0->L;
  g->B = count;
  g->C = ((2 * count + kBN - 1) / kBN) * kBN;
  g->p = p0->p;
  g->terms = p0->terms;
  g->mode = mode;
  g->stream = p0->stream;
  const size_t L = size_t(g->L), LB = L * count, LL = L * L, LC = L * size_t(g->C);
  const bool bf16 = (mode == PE_GEMM_BF16X3), split = (mode == PE_GEMM_BF16X3 || mode == PE_GEMM_3XTF32);
  const size_t el = bf16 ? 2 : 4;
  auto bail = [&](const char* what) {
    p0->err = std::string("GEMM batch: ") + what;
    pe_gemm_batch_destroy(g);
    return PE_ERR_CUDA;
  };
  float* S32 = nullptr;
  if (cudaMalloc(&S32, sizeof(float) * LL) != cudaSuccess) return bail("cudaMalloc");
  const size_t planes = split ? 2 : 1;  // hi and lo parts back to back (one allocation each)
  bool okm = cudaMalloc(&g->Shi, planes * el * LL) == cudaSuccess && cudaMalloc(&g->Y, sizeof(float2) * LB) == cudaSuccess &&
             cudaMalloc(&g->ACC, sizeof(float2) * LB) == cudaSuccess &&
             cudaMalloc(&g->G, sizeof(float) * LC) == cudaSuccess &&
             cudaMalloc(&g->dSolves, sizeof(GemmSolve) * count) == cudaSuccess &&
             cudaMalloc(&g->status, sizeof(int)) == cudaSuccess;
  for (int b = 0; b < 2 && okm; ++b) okm = cudaMalloc(&g->Xhi[b], planes * el * LC) == cudaSuccess;
  if (okm && split) {
    g->Slo = static_cast<uint8_t*>(g->Shi) + el * LL;
    for (int b = 0; b < 2; ++b) g->Xlo[b] = static_cast<uint8_t*>(g->Xhi[b]) + el * LC;
  }
  if (!okm) {
    cudaFree(S32);
    return bail("cudaMalloc");
  }
  for (int b = 0; b < 2; ++b) cudaMemset(g->Xhi[b], 0, planes * el * LC);  // padding columns must read as zero
  cudaMemset(g->status, 0, sizeof(int));
  // the DST-I matrix in FP64, rounded once (symmetric; row and column 0 are the zero pads)
  std::vector<float> S(LL);
  for (size_t m = 0; m < L; ++m)
    for (size_t n = 0; n < L; ++n) {
      const size_t q = (m * n) % (2 * L);
      S[m * L + n] = float(std::sin(M_PI * double(q) / double(L)));
    }
  if (cudaMemcpy(S32, S.data(), sizeof(float) * LL, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(S32);
    return bail("upload");
  }
  k_split_s<<<int((LL + 255) / 256), 256, 0, g->stream>>>(S32, g->Shi, g->Slo, LL, mode);
  cudaStreamSynchronize(g->stream);
  cudaFree(S32);
  if (cudaGetLastError() != cudaSuccess) return bail("split");
  if (mode != PE_GEMM_FP32) {
    bool okt = make_map(&g->mS, g->Shi, bf16, L, L, kBM, int(planes), el * LL);
    for (int b = 0; b < 2 && okt; ++b)
      okt = make_map(&g->mX[b], g->Xhi[b], bf16, L, size_t(g->C), kBN, int(planes), el * LC);
    if (!okt) return bail("tensor map (cuTensorMapEncodeTiled)");
  }
  std::vector<GemmSolve> sv(count);
  std::vector<const float2*> yh(count);
  for (int i = 0; i < count; ++i) {
    sv[i].A = plans[i]->dA;
    sv[i].B = plans[i]->dB;
    sv[i].R = plans[i]->dR;
    sv[i].V = plans[i]->dV;
    for (int j = 0; j < sssp::kMaxStages; ++j) sv[i].beta[j] = plans[i]->beta[j];
    yh[i] = plans[i]->dYhat;
  }
  if (cudaMemcpy(g->dSolves, sv.data(), sizeof(GemmSolve) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail("upload");
  const float2** dyh = nullptr;
  if (cudaMalloc(&dyh, sizeof(float2*) * count) != cudaSuccess) return bail("cudaMalloc");
  cudaMemcpy(dyh, yh.data(), sizeof(float2*) * count, cudaMemcpyHostToDevice);
  k_gather<<<int((LB + 255) / 256), 256, 0, g->stream>>>(dyh, g->Y, g->L, count);
  cudaStreamSynchronize(g->stream);
  cudaFree(dyh);
  if (cudaGetLastError() != cudaSuccess) return bail("gather");
  for (int i = 0; i < count; ++i) g->sigma.push_back(plans[i]->k0 * plans[i]->dr);
  // one range step as a CUDA graph
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bail("stream");
  cudaStream_t keep = g->stream;
  g->stream = cap;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return bail("capture");
  pe_status st = enqueue_step(g);
  if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || st != PE_OK) return bail("capture");
  if (cudaGraphInstantiate(&g->step_graph, graph, 0) != cudaSuccess) return bail("instantiate");
  cudaGraphDestroy(graph);
  g->stream = keep;
  cudaStreamDestroy(cap);
  *out = g;
  return PE_OK;
}

pe_status pe_gemm_batch_march(pe_gemm_batch* g, int steps) {
  if (!g || steps < 0) return PE_ERR_ARG;
  for (int s = 0; s < steps; ++s)
    if (cudaGraphLaunch(g->step_graph, g->stream) != cudaSuccess) return gfail(g, PE_ERR_CUDA, "graph launch");
  g->steps_done += steps;
  return PE_OK;
}

pe_status pe_gemm_batch_read_field(pe_gemm_batch* g, int index, float* out) {
  if (!g || !out || index < 0 || index >= g->B) return PE_ERR_ARG;
  ElemArgs a = elem_args(g, 0, 0);
  a.scale = float(2.0 / double(g->L));
  stage_out(g, a);
  const unsigned long long keep = g->gemms_per_step;
  cudaError_t e = launch_gemm(g, kEpiOut, 0, 0);
  g->gemms_per_step = keep;
  if (e != cudaSuccess) return gfail(g, PE_ERR_CUDA, std::string("GEMM launch: ") + cudaGetErrorString(e));
  std::vector<float> re(g->L), im(g->L);
  int status = 0;
  cudaMemcpyAsync(re.data(), g->G + size_t(2 * index) * g->L, sizeof(float) * g->L, cudaMemcpyDeviceToHost, g->stream);
  cudaMemcpyAsync(im.data(), g->G + size_t(2 * index + 1) * g->L, sizeof(float) * g->L, cudaMemcpyDeviceToHost,
                  g->stream);
  cudaMemcpyAsync(&status, g->status, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return gfail(g, PE_ERR_CUDA, "sync");
  if (status != 0) return gfail(g, PE_ERR_TIMEOUT, "GEMM kernel: a barrier wait ran out (device status set)");
  const double ph = std::fmod(g->sigma[index] * double(g->steps_done), 2.0 * M_PI);
  const double c = std::cos(ph), s = std::sin(ph);
  for (int n = 0; n < g->N; ++n) {  // depth index n + 1 of the L-indexed output
    out[2 * n] = float(c * re[n + 1] - s * im[n + 1]);
    out[2 * n + 1] = float(c * im[n + 1] + s * re[n + 1]);
  }
  return PE_OK;
}

const char* pe_gemm_batch_error(const pe_gemm_batch* g) { return g ? g->err.c_str() : ""; }

void pe_gemm_batch_destroy(pe_gemm_batch* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->step_graph) cudaGraphExecDestroy(g->step_graph);
  cudaFree(g->dSolves);
  cudaFree(g->Shi);  // the lo planes live in the same allocations
  for (int b = 0; b < 2; ++b) cudaFree(g->Xhi[b]);
  cudaFree(g->Y);
  cudaFree(g->ACC);
  cudaFree(g->G);
  cudaFree(g->status);
  delete g;
}

}  // extern "C"
