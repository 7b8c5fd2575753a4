// Batched march with the DST-I as a dense GEMM on the tensor cores (a precision variant).
//
// For a batch of B solves of one grid size, every transform of the march is applied to all B
// fields at once as Y = S X, S[m][n] = sin(pi n m/(N+1)) (N x N, real, symmetric) and X the
// N x 2B real matrix of the fields' real and imaginary parts.  The GEMM is a plain library
// contraction (cuBLAS) in one of four precisions:
//   PE_GEMM_FP32    FP32 on the CUDA cores (reference for the others),
//   PE_GEMM_TF32    one TF32 tensor-core GEMM,
//   PE_GEMM_3XTF32  S = S_hi + S_lo, X = X_hi + X_lo (TF32 hi parts): S_hi X_hi + S_hi X_lo + S_lo X_hi,
//   PE_GEMM_BF16X3  the same split with BF16 parts,
// all accumulating in FP32.  Everything else of the step (Pade multipliers, V multiply,
// Neumann accumulation, stage update with hi/lo multipliers) runs in this file's element-wise
// kernels, with the same tables and arithmetic as the FFT marcher.  The series takes a fixed
// number of terms (the plans' neumann_terms) for every solve, so all solves stay in lockstep;
// one range step is captured once in a CUDA graph and replayed.
//
// The dense transform costs 4 N^2 flop per complex vector against ~5 (N+1) log2(N+1) for the
// FFT (about 80x more at N = 1023), so this form is measured for its accuracy per precision,
// not offered as the fast path.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sssp.h"
#include "plan_internal.h"

namespace {

struct GemmSolve {  // per-solve table pointers (device)
  const float2* A;
  const float2* B;
  const float4* R;
  const float* V;
  float2 beta[sssp::kMaxStages];
};

__device__ __forceinline__ float tf32_hi(float x) {
  // round to the nearest value with a 10-bit mantissa (TF32), ties away
  unsigned u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// writes the GEMM input columns (re in column b, im in column B + b) in the chosen precision
__device__ __forceinline__ void put_x(float* xf, __nv_bfloat16* xh, __nv_bfloat16* xl, float* xlo, int mode, size_t ir,
                                      size_t ii, float2 v) {
  if (mode == PE_GEMM_BF16X3) {
    const __nv_bfloat16 hr = __float2bfloat16(v.x), hi = __float2bfloat16(v.y);
    xh[ir] = hr;
    xh[ii] = hi;
    xl[ir] = __float2bfloat16(v.x - __bfloat162float(hr));
    xl[ii] = __float2bfloat16(v.y - __bfloat162float(hi));
  } else if (mode == PE_GEMM_3XTF32) {
    const float hr = tf32_hi(v.x), hi = tf32_hi(v.y);
    xf[ir] = hr;
    xf[ii] = hi;
    xlo[ir] = v.x - hr;
    xlo[ii] = v.y - hi;
  } else {
    xf[ir] = v.x;
    xf[ii] = v.y;
  }
}

struct Args {
  const GemmSolve* solves;
  float2* Y;      // N x B spectral state (complex, row n = mode n+1, column b)
  float2* T0;     // N x B
  float2* ACC;    // N x B
  const float* G; // N x 2B GEMM output (real columns)
  float* XF;      // GEMM input, FP32 / TF32 hi
  float* XLO;     // TF32 lo
  __nv_bfloat16* XH;
  __nv_bfloat16* XL;
  int N, B, mode, j;
};

// stage start: t0 = A_j y (spectral), acc = 0, X <- t0
__global__ void k_stage_start(Args a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(a.N) * a.B) return;
  const int n = int(idx % a.N), b = int(idx / a.N);
  const GemmSolve& s = a.solves[b];
  const size_t L = size_t(a.N) + 1;
  const float2 Av = s.A[size_t(a.j) * L + n + 1], y = a.Y[idx];
  const float2 t0 = make_float2(fmaf(Av.x, y.x, -Av.y * y.y), fmaf(Av.x, y.y, Av.y * y.x));
  a.T0[idx] = t0;
  a.ACC[idx] = make_float2(0.f, 0.f);
  put_x(a.XF, a.XH, a.XL, a.XLO, a.mode, size_t(b) * a.N + n, size_t(a.B + b) * a.N + n, t0);
}

// depth space: X <- V .* (GEMM output)
__global__ void k_times_v(Args a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(a.N) * a.B) return;
  const int n = int(idx % a.N), b = int(idx / a.N);
  const float v = a.solves[b].V[n + 1];
  const size_t ir = size_t(b) * a.N + n, ii = size_t(a.B + b) * a.N + n;
  put_x(a.XF, a.XH, a.XL, a.XLO, a.mode, ir, ii, make_float2(v * a.G[ir], v * a.G[ii]));
}

// spectral: t_m = B_j .* (GEMM output); acc += t_m; X <- t_m
__global__ void k_term(Args a, int write_x) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(a.N) * a.B) return;
  const int n = int(idx % a.N), b = int(idx / a.N);
  const size_t L = size_t(a.N) + 1;
  const float2 Bv = a.solves[b].B[size_t(a.j) * L + n + 1];
  const size_t ir = size_t(b) * a.N + n, ii = size_t(a.B + b) * a.N + n;
  const float2 u = make_float2(a.G[ir], a.G[ii]);
  const float2 th = make_float2(fmaf(Bv.x, u.x, -Bv.y * u.y), fmaf(Bv.x, u.y, Bv.y * u.x));
  const float2 acc = a.ACC[idx];
  a.ACC[idx] = make_float2(acc.x + th.x, acc.y + th.y);
  if (write_x) put_x(a.XF, a.XH, a.XL, a.XLO, a.mode, ir, ii, th);
}

// stage end: y = R_j y (hi/lo multiplier) + beta_j acc
__global__ void k_stage_end(Args a) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(a.N) * a.B) return;
  const int n = int(idx % a.N), b = int(idx / a.N);
  const GemmSolve& s = a.solves[b];
  const size_t L = size_t(a.N) + 1;
  const float4 g = s.R[size_t(a.j) * L + n + 1];
  const float2 y = a.Y[idx], acc = a.ACC[idx], bj = s.beta[a.j];
  const float re_lo = fmaf(g.z, y.x, -g.w * y.y), im_lo = fmaf(g.z, y.y, g.w * y.x);
  const float re = fmaf(g.x, y.x, fmaf(-g.y, y.y, re_lo)), im = fmaf(g.x, y.y, fmaf(g.y, y.x, im_lo));
  a.Y[idx] = make_float2(re + fmaf(bj.x, acc.x, -bj.y * acc.y), im + fmaf(bj.x, acc.y, bj.y * acc.x));
}

// X <- scale * Y (for the final depth-space field)
__global__ void k_out(Args a, float scale) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(a.N) * a.B) return;
  const int n = int(idx % a.N), b = int(idx / a.N);
  const float2 y = a.Y[idx];
  put_x(a.XF, a.XH, a.XL, a.XLO, a.mode, size_t(b) * a.N + n, size_t(a.B + b) * a.N + n,
        make_float2(scale * y.x, scale * y.y));
}

__global__ void k_split_s(const float* S, float* shi, float* slo, __nv_bfloat16* bh, __nv_bfloat16* bl, size_t n,
                          int mode) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = S[i];
  if (mode == PE_GEMM_BF16X3) {
    const __nv_bfloat16 h = __float2bfloat16(v);
    bh[i] = h;
    bl[i] = __float2bfloat16(v - __bfloat162float(h));
  } else if (mode == PE_GEMM_3XTF32) {
    const float h = tf32_hi(v);
    shi[i] = h;
    slo[i] = v - h;
  }
}

// gather the spectral states of the plans (mode index 1..N) into Y
__global__ void k_gather(const float2* const* yhats, float2* Y, int N, int B) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(N) * B) return;
  const int n = int(idx % N), b = int(idx / N);
  Y[idx] = yhats[b][n + 1];
}

}  // namespace

struct pe_gemm_batch {
  int N = 0, B = 0, p = 0, terms = 0, mode = 0;
  std::vector<double> sigma;  // k0 dr of every member (the carrier phase per step)
  long long steps_done = 0;
  cudaStream_t stream = nullptr;
  cublasHandle_t h = nullptr;
  void* ws = nullptr;
  GemmSolve* dSolves = nullptr;
  float* S = nullptr;  // N x N FP32
  float* Shi = nullptr;
  float* Slo = nullptr;
  __nv_bfloat16* Sbh = nullptr;
  __nv_bfloat16* Sbl = nullptr;
  float2 *Y = nullptr, *T0 = nullptr, *ACC = nullptr;
  float *G = nullptr, *XF = nullptr, *XLO = nullptr;
  __nv_bfloat16 *XH = nullptr, *XL = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  std::string err;
};

namespace {

pe_status gfail(pe_gemm_batch* g, pe_status s, const std::string& m) {
  if (g) g->err = m;
  return s;
}

// G = S X in the batch's precision
cublasStatus_t gemm(pe_gemm_batch* g) {
  const int m = g->N, n = 2 * g->B, k = g->N;
  const float one = 1.f, zero = 0.f;
  switch (g->mode) {
    case PE_GEMM_FP32:
      return cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->S, CUDA_R_32F, m, g->XF, CUDA_R_32F, k,
                          &zero, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_PEDANTIC, CUBLAS_GEMM_DEFAULT);
    case PE_GEMM_TF32:
      return cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->S, CUDA_R_32F, m, g->XF, CUDA_R_32F, k,
                          &zero, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT);
    case PE_GEMM_3XTF32: {
      cublasStatus_t s = cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Shi, CUDA_R_32F, m, g->XF,
                                      CUDA_R_32F, k, &zero, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_FAST_TF32,
                                      CUBLAS_GEMM_DEFAULT);
      if (s != CUBLAS_STATUS_SUCCESS) return s;
      s = cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Shi, CUDA_R_32F, m, g->XLO, CUDA_R_32F, k,
                       &one, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT);
      if (s != CUBLAS_STATUS_SUCCESS) return s;
      return cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Slo, CUDA_R_32F, m, g->XF, CUDA_R_32F, k,
                          &one, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT);
    }
    case PE_GEMM_BF16X3: {
      cublasStatus_t s = cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Sbh, CUDA_R_16BF, m, g->XH,
                                      CUDA_R_16BF, k, &zero, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F,
                                      CUBLAS_GEMM_DEFAULT);
      if (s != CUBLAS_STATUS_SUCCESS) return s;
      s = cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Sbh, CUDA_R_16BF, m, g->XL, CUDA_R_16BF, k,
                       &one, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
      if (s != CUBLAS_STATUS_SUCCESS) return s;
      return cublasGemmEx(g->h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, g->Sbl, CUDA_R_16BF, m, g->XH, CUDA_R_16BF,
                          k, &one, g->G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    }
  }
  return CUBLAS_STATUS_INVALID_VALUE;
}

Args args_of(pe_gemm_batch* g, int j) {
  Args a;
  a.solves = g->dSolves;
  a.Y = g->Y;
  a.T0 = g->T0;
  a.ACC = g->ACC;
  a.G = g->G;
  a.XF = g->XF;
  a.XLO = g->XLO;
  a.XH = g->XH;
  a.XL = g->XL;
  a.N = g->N;
  a.B = g->B;
  a.mode = g->mode;
  a.j = j;
  return a;
}

// enqueue one range step (all stages, fixed term count) on g->stream
pe_status enqueue_step(pe_gemm_batch* g) {
  const size_t tot = size_t(g->N) * g->B;
  const int th = 256, bl = int((tot + th - 1) / th);
  for (int j = 0; j < g->p; ++j) {
    Args a = args_of(g, j);
    k_stage_start<<<bl, th, 0, g->stream>>>(a);
    if (gemm(g) != CUBLAS_STATUS_SUCCESS) return gfail(g, PE_ERR_CUDA, "cuBLAS GEMM failed");  // t_0 in depth space
    for (int m = 1; m < g->terms; ++m) {
      k_times_v<<<bl, th, 0, g->stream>>>(a);
      if (gemm(g) != CUBLAS_STATUS_SUCCESS) return gfail(g, PE_ERR_CUDA, "cuBLAS GEMM failed");  // DST(V t)
      const int last = (m == g->terms - 1);
      k_term<<<bl, th, 0, g->stream>>>(a, last ? 0 : 1);
      if (!last && gemm(g) != CUBLAS_STATUS_SUCCESS) return gfail(g, PE_ERR_CUDA, "cuBLAS GEMM failed");
    }
    k_stage_end<<<bl, th, 0, g->stream>>>(a);
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
  for (int i = 0; i < count; ++i) {
    pe_plan* p = plans[i];
    if (!p || p->N != p0->N || p->p != p0->p || p->terms != p0->terms || p->dr != p0->dr) {
      if (p0) p0->err = "GEMM batch: plans must share N, Pade order, term count and dr";
      return PE_ERR_ARG;
    }
    if (!p->field_set || p->terms < 2 || p->nodes != 1 || p->complex_profile || p->bc != PE_BC_DIRICHLET) {
      p0->err = "GEMM batch: every plan needs a field, one real profile node and neumann_terms >= 2";
      return PE_ERR_STATE;
    }
  }
  pe_gemm_batch* g = new pe_gemm_batch();
  g->N = p0->N;
  g->B = count;
  g->p = p0->p;
  g->terms = p0->terms;
  g->mode = mode;
  g->stream = p0->stream;
  const size_t N = size_t(g->N), NB = N * count, NN = N * N;
  auto bail = [&](const char* what) {
    p0->err = std::string("GEMM batch: ") + what;
    pe_gemm_batch_destroy(g);
    return PE_ERR_CUDA;
  };
  if (cublasCreate(&g->h) != CUBLAS_STATUS_SUCCESS) return bail("cublasCreate");
  cublasSetStream(g->h, g->stream);
  const size_t ws_bytes = size_t(32) << 20;
  if (cudaMalloc(&g->ws, ws_bytes) != cudaSuccess) return bail("workspace");
  cublasSetWorkspace(g->h, g->ws, ws_bytes);
  if (cudaMalloc(&g->S, sizeof(float) * NN) != cudaSuccess || cudaMalloc(&g->Y, sizeof(float2) * NB) != cudaSuccess ||
      cudaMalloc(&g->T0, sizeof(float2) * NB) != cudaSuccess || cudaMalloc(&g->ACC, sizeof(float2) * NB) != cudaSuccess ||
      cudaMalloc(&g->G, sizeof(float) * 2 * NB) != cudaSuccess || cudaMalloc(&g->XF, sizeof(float) * 2 * NB) != cudaSuccess ||
      cudaMalloc(&g->dSolves, sizeof(GemmSolve) * count) != cudaSuccess)
    return bail("cudaMalloc");
  if (mode == PE_GEMM_3XTF32 &&
      (cudaMalloc(&g->Shi, sizeof(float) * NN) != cudaSuccess || cudaMalloc(&g->Slo, sizeof(float) * NN) != cudaSuccess ||
       cudaMalloc(&g->XLO, sizeof(float) * 2 * NB) != cudaSuccess))
    return bail("cudaMalloc");
  if (mode == PE_GEMM_BF16X3 &&
      (cudaMalloc(&g->Sbh, sizeof(__nv_bfloat16) * NN) != cudaSuccess ||
       cudaMalloc(&g->Sbl, sizeof(__nv_bfloat16) * NN) != cudaSuccess ||
       cudaMalloc(&g->XH, sizeof(__nv_bfloat16) * 2 * NB) != cudaSuccess ||
       cudaMalloc(&g->XL, sizeof(__nv_bfloat16) * 2 * NB) != cudaSuccess))
    return bail("cudaMalloc");
  // the DST-I matrix in FP64, rounded once (symmetric, so row/column order does not matter)
  std::vector<float> S(NN);
  const long long L = (long long)N + 1;
  for (size_t m = 1; m <= N; ++m)
    for (size_t n = 1; n <= N; ++n) {
      const long long q = (long long)((m * n) % size_t(2 * L));
      S[(m - 1) * N + (n - 1)] = float(std::sin(M_PI * double(q) / double(L)));
    }
  if (cudaMemcpy(g->S, S.data(), sizeof(float) * NN, cudaMemcpyHostToDevice) != cudaSuccess) return bail("upload");
  if (mode == PE_GEMM_3XTF32 || mode == PE_GEMM_BF16X3) {
    k_split_s<<<int((NN + 255) / 256), 256, 0, g->stream>>>(g->S, g->Shi, g->Slo, g->Sbh, g->Sbl, NN, mode);
    if (cudaGetLastError() != cudaSuccess) return bail("split");
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
  k_gather<<<int((NB + 255) / 256), 256, 0, g->stream>>>(dyh, g->Y, g->N, count);
  cudaStreamSynchronize(g->stream);
  cudaFree(dyh);
  if (cudaGetLastError() != cudaSuccess) return bail("gather");
  for (int i = 0; i < count; ++i) g->sigma.push_back(plans[i]->k0 * plans[i]->dr);
  // one range step as a CUDA graph (cuBLAS runs on the user workspace, so it can be captured)
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bail("stream");
  cudaStream_t keep = g->stream;
  g->stream = cap;
  cublasSetStream(g->h, cap);
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return bail("capture");
  pe_status st = enqueue_step(g);
  if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || st != PE_OK) return bail("capture");
  if (cudaGraphInstantiate(&g->step_graph, graph, 0) != cudaSuccess) return bail("instantiate");
  cudaGraphDestroy(graph);
  g->stream = keep;
  cublasSetStream(g->h, keep);
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
  Args a = args_of(g, 0);
  const size_t tot = size_t(g->N) * g->B;
  k_out<<<int((tot + 255) / 256), 256, 0, g->stream>>>(a, float(2.0 / double(g->N + 1)));
  if (gemm(g) != CUBLAS_STATUS_SUCCESS) return gfail(g, PE_ERR_CUDA, "cuBLAS GEMM failed");
  std::vector<float> re(g->N), im(g->N);
  cudaMemcpyAsync(re.data(), g->G + size_t(index) * g->N, sizeof(float) * g->N, cudaMemcpyDeviceToHost, g->stream);
  cudaMemcpyAsync(im.data(), g->G + size_t(g->B + index) * g->N, sizeof(float) * g->N, cudaMemcpyDeviceToHost,
                  g->stream);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return gfail(g, PE_ERR_CUDA, "sync");
  const double ph = std::fmod(g->sigma[index] * double(g->steps_done), 2.0 * M_PI);
  const double c = std::cos(ph), s = std::sin(ph);
  for (int n = 0; n < g->N; ++n) {
    out[2 * n] = float(c * re[n] - s * im[n]);
    out[2 * n + 1] = float(c * im[n] + s * re[n]);
  }
  return PE_OK;
}

const char* pe_gemm_batch_error(const pe_gemm_batch* g) { return g ? g->err.c_str() : ""; }

void pe_gemm_batch_destroy(pe_gemm_batch* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->step_graph) cudaGraphExecDestroy(g->step_graph);
  if (g->h) cublasDestroy(g->h);
  cudaFree(g->ws);
  cudaFree(g->dSolves);
  cudaFree(g->S);
  cudaFree(g->Shi);
  cudaFree(g->Slo);
  cudaFree(g->Sbh);
  cudaFree(g->Sbl);
  cudaFree(g->Y);
  cudaFree(g->T0);
  cudaFree(g->ACC);
  cudaFree(g->G);
  cudaFree(g->XF);
  cudaFree(g->XLO);
  cudaFree(g->XH);
  cudaFree(g->XL);
  delete g;
}

}  // extern "C"
