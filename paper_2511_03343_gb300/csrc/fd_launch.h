// Internal interface of the FD-SSP march (march_fd.cuh): launch and host factorisation.
#pragma once
#include <cuda_runtime.h>

#include <complex>

namespace sssp {
struct SolveDesc;
}

namespace sssp_fd {

bool supported(int log2L);  // L = N + 1 in [8, 4096]
cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st);
// FP64 Thomas factors of 1 + b_j X, X = D2/k0^2 + V, for every stage j of one profile node
// (V: N values, n = 1..N), as the kernel's table entries: out gets p x L x 3 float4 (index 0 the
// boundary)
void factor_node(const double* V, int N, int L, double H, double k0, const std::complex<double>* b, int p,
                 float4* out);

}  // namespace sssp_fd
