// Internal layout of pe_plan, shared by the translation units of the library (not part of
// the C ABI: callers only see the opaque handle).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "march_kernel.cuh"
#include "pade_host.h"

struct TransformTables {
  float2* tw = nullptr;  // per-pass Stockham twiddles (L - 8 used entries)
  float* sinw = nullptr; // L weights sin(pi n/L)
};

struct pe_plan {
  int N = 0, L = 0, log2L = 0, p = 0, terms = 0, device = 0;
  int bc = 0;   // transform the kernels run: PE_BC_DIRICHLET or PE_BC_PERIODIC
  int user_bc = 0;  // the caller's boundary condition (PE_BC_NEUMANN runs as a periodic plan on
                    // the even extension of the field to [0, 2H])
  int N_user = 0;   // grid points the caller sees
  int kernel = 0;   // PE_KERNEL_AUTO / PE_KERNEL_CTA / PE_KERNEL_CLUSTER
  int ppt = 8;      // points per thread of the one-CTA kernel (4, 8 or 16; pe_plan_set_shape)
  int cl_ncta = 0;  // cluster kernel shape: CTAs per cluster (0: the size's default) and
  int cl_push = -1; // exchange by remote stores 1 / loads 0 (-1: default; pe_plan_set_cluster_shape)
  int op = 0;       // PE_OP_SPECTRAL (the paper's DST-I operator) or PE_OP_FD3 (FD-SSP)
  float4* dFD = nullptr;   // FD-SSP: node_cap x p x L x 3 float4 Thomas factors (hi + lo)
  float4* dFDc = nullptr;  // FD-SSP: per stage hi/lo of a_j/b_j and 1 - a_j/b_j
  int fd_cap = 0;          // nodes dFD holds
  double cost = 0.0;       // DST-I per range step measured by the batch autotuner (0: unknown);
                           // a batched launch orders its solves by it
  int off = 1;  // index of the first stored depth point in the length-L arrays
  double H = 0, k0 = 0, dr = 0, tol = 0;
  cudaStream_t stream = nullptr;
  sssp::PadeData pade;
  TransformTables tabs;
  float4* dR = nullptr;
  float2* dA = nullptr;
  float2* dB = nullptr;
  float4* dG = nullptr;
  float2 beta[sssp::kMaxStages];
  float2* dYhat = nullptr;
  float2* dField = nullptr;
  float2* dStage = nullptr;  // N-value staging buffer (set / read field)
  float2* dWork = nullptr;   // 4 L workspace for grids beyond one CTA's shared memory
  float* dV = nullptr;
  float* dVi = nullptr;      // imaginary parts of n^2, allocated with the first complex node
  bool complex_profile = false;
  double* dNodeR = nullptr;
  int nodes = 0, node_cap = 0;
  std::vector<double> node_r;
  int* dStatus = nullptr;
  unsigned long long* dNdst = nullptr;
  float* dTL = nullptr;
  long long tl_cap_rows = 0, tl_rows = 0;
  std::vector<double> tl_ranges;
  int tl_every = 0;
  sssp::SolveDesc* dDesc = nullptr;
  size_t desc_cap = 0;  // bytes of dDesc (batched marches led by this plan reuse it)
  double r_set = 0.0;
  long long steps_done = 0;
  bool field_set = false;
  std::string err;
};

