// FD-SSP range march (the comparison of Section 4.3): the product-form Pade propagator of
// Section 2 with the standard 3-point finite difference for d_z^2 (our choice of stencil),
// X = D2/k0^2 + V, D2 u_n = (u_{n+1} - 2 u_n + u_{n-1})/dz^2, Dirichlet boundaries.  Each stage
// solves (1 + b_j X) w = y directly and sets y <- (a_j/b_j) y + (1 - a_j/b_j) w.
//
// The tridiagonal matrix 1 + b_j X (diagonal 1 + b_j(V_n - 2 s), off-diagonals e_j = b_j s,
// s = 1/(k0 dz)^2) is factored once per profile node and stage on the host in FP64 (no
// pivoting, as the usual FD-SSP marchers do): with c'_n the Thomas multipliers and inv_n the
// inverted pivots, the forward sweep is g_n = inv_n y_n - e_j inv_n g_{n-1} and the back sweep
// w_n = g_n - c'_n w_{n+1}.  Both are first-order linear recurrences, so each runs as one
// block-wide scan of affine maps x -> alpha x + beta (composition is associative): every thread
// composes its 8 consecutive points, a warp shuffle scan and a scan over the warps combine the
// chunks, then each thread replays its points from its prefix.  The field stays in registers
// (thread t owns depth indices 8t .. 8t + 7; index 0 is the zero boundary) for all range steps.
// The table constants are hi + lo pairs, so their FP32 representation error does not add up
// coherently over the steps.
#pragma once
#include "march_kernel.cuh"

namespace sssp {

constexpr int kFdMinLog2 = 3;
constexpr int kFdMaxLog2 = 12;

// one table entry per point and stage: inv_n, alpha_n = -e_j inv_n, -c'_n (each hi + lo)
struct FdEntry {
  float4 inv, alpha, mcp;
};

template <int LOG2L>
struct FdCfg {
  static constexpr int L = 1 << LOG2L;
  static constexpr int PT = 8;
  static constexpr int NT = L / PT;
  static constexpr int WS = NT >= 32 ? 32 : NT;
  static constexpr int NW = (NT + 31) / 32;
  static constexpr unsigned MASK = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
};

// affine map x -> a x + b, a and b complex
struct Aff {
  float2 a, b;
};

// the map "first f, then g"
__device__ __forceinline__ Aff aff_then(const Aff& f, const Aff& g) {
  return Aff{cmul(g.a, f.a), cmul(g.a, f.b) + g.b};
}

__device__ __forceinline__ Aff aff_shfl_up(const Aff& v, int o, unsigned mask, int ws) {
  return Aff{make_float2(__shfl_up_sync(mask, v.a.x, o, ws), __shfl_up_sync(mask, v.a.y, o, ws)),
             make_float2(__shfl_up_sync(mask, v.b.x, o, ws), __shfl_up_sync(mask, v.b.y, o, ws))};
}
__device__ __forceinline__ Aff aff_shfl_down(const Aff& v, int o, unsigned mask, int ws) {
  return Aff{make_float2(__shfl_down_sync(mask, v.a.x, o, ws), __shfl_down_sync(mask, v.a.y, o, ws)),
             make_float2(__shfl_down_sync(mask, v.b.x, o, ws), __shfl_down_sync(mask, v.b.y, o, ws))};
}

// The map applied before thread t's chunk, in scan order (ascending thread index if !REV, else
// descending), given the thread's own chunk map `own`.  sh: 2 NW Aff of shared memory.  Every
// thread must call it.
template <int LOG2L, bool REV>
__device__ __forceinline__ Aff block_prefix(const Aff& own, Aff* sh) {
  using C = FdCfg<LOG2L>;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // inclusive scan within the warp: lanes earlier in scan order come first
  Aff inc = own;
#pragma unroll
  for (int o = 1; o < C::WS; o <<= 1) {
    const Aff e = REV ? aff_shfl_down(inc, o, C::MASK, C::WS) : aff_shfl_up(inc, o, C::MASK, C::WS);
    const bool has = REV ? (lane + o < C::WS) : (lane >= o);
    if (has) inc = aff_then(e, inc);
  }
  Aff excl = REV ? aff_shfl_down(inc, 1, C::MASK, C::WS) : aff_shfl_up(inc, 1, C::MASK, C::WS);
  if (REV ? (lane == C::WS - 1) : (lane == 0)) excl = Aff{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
  if constexpr (C::NW > 1) {
    __syncthreads();  // earlier users of sh are done
    if (REV ? (lane == 0) : (lane == C::WS - 1)) sh[warp] = inc;  // the warp's total map
    __syncthreads();
    Aff off{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
    if (REV) {
      for (int w = C::NW - 1; w > warp; --w) off = aff_then(off, sh[w]);
    } else {
      for (int w = 0; w < warp; ++w) off = aff_then(off, sh[w]);
    }
    excl = aff_then(off, excl);
  }
  return excl;
}

template <int LOG2L>
__global__ void __launch_bounds__(FdCfg<LOG2L>::NT)
    sssp_fd_march_kernel(const SolveDesc* __restrict__ descs) {
  using C = FdCfg<LOG2L>;
  constexpr int L = C::L, P = C::PT;
  __shared__ SolveDesc d;
  __shared__ Aff sh[2 * C::NW];
  const int t = threadIdx.x;
  {
    const int* src = reinterpret_cast<const int*>(descs + blockIdx.x);
    int* dst = reinterpret_cast<int*>(&d);
    for (int i = t; i < int(sizeof(SolveDesc) / sizeof(int)); i += C::NT) dst[i] = src[i];
  }
  __syncthreads();
  float2 y[P];
  load8<LOG2L, P>(d.yhat + P * t, y);  // depth values (index 0: the boundary, 0)
  int node = d.node0;
  double next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
  int nrec = 0;
  for (int s = 0; s < d.steps; ++s) {
    const double rmid = d.r0 + (double(s) + 0.5) * d.dr;
    if (rmid >= next_r) {
      while (node + 1 < d.nodes && d.node_r[node + 1] <= rmid) ++node;
      next_r = (node + 1 < d.nodes) ? d.node_r[node + 1] : 1e300;
    }
    for (int j = 0; j < d.p; ++j) {
      const FdEntry* tab = reinterpret_cast<const FdEntry*>(d.fd) + ((size_t)node * d.p + j) * L + P * t;
      // forward sweep g_n = alpha_n g_{n-1} + inv_n y_n
      float2 be[P];
      Aff own{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const FdEntry e = tab[i];
        be[i] = ffmul(e.inv, y[i]);
        own = Aff{ffmul(e.alpha, own.a), ffmul(e.alpha, own.b) + be[i]};
      }
      Aff pre = block_prefix<LOG2L, false>(own, sh);
      float2 x = pre.b;  // the sweep starts from g = 0 before index 0
      float2 g[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        x = ffmul(tab[i].alpha, x) + be[i];
        g[i] = x;
      }
      // back sweep w_n = -c'_n w_{n+1} + g_n (descending n)
      Aff own2{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
      for (int i = P - 1; i >= 0; --i) {
        const float4 m = tab[i].mcp;
        own2 = Aff{ffmul(m, own2.a), ffmul(m, own2.b) + g[i]};
      }
      Aff pre2 = block_prefix<LOG2L, true>(own2, sh + C::NW);
      float2 w = pre2.b;  // w = 0 beyond the last point
      const float4 c1 = d.fdc[2 * j], c2 = d.fdc[2 * j + 1];
#pragma unroll
      for (int i = P - 1; i >= 0; --i) {
        w = ffmul(tab[i].mcp, w) + g[i];
        y[i] = ffmul(c1, y[i]) + ffmul(c2, w);  // (a_j/b_j) y + (1 - a_j/b_j) w
      }
    }
    const long long gs = d.step0 + s + 1;
    if (d.tl_every > 0 && gs % d.tl_every == 0) {
      const float lr = float(10.0 * log10(d.r0 + double(s + 1) * d.dr));
      float* row = d.tl + (size_t)(d.rec0 + nrec) * d.N;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int n = P * t + i;
        if (n >= 1) row[n - 1] = fmaf(-10.f, log10f(cabs2(y[i])), lr);
      }
      ++nrec;
    }
  }
  store8<LOG2L, P>(d.yhat + P * t, y);
  store8<LOG2L, P>(d.field + P * t, y);
}

}  // namespace sssp
