// Launch of the FD-SSP march kernel (march_fd.cuh), L = N + 1 = 8 .. 4096, and the host FP64
// factorisation of its tridiagonal stage matrices.
#include <cuda_runtime.h>

#include <complex>
#include <vector>

#include "fd_launch.h"
#include "march_fd.cuh"

namespace sssp_fd {

namespace {

template <int LOG2L>
cudaError_t launch_t(const sssp::SolveDesc* d, int count, cudaStream_t st) {
  sssp::sssp_fd_march_kernel<LOG2L><<<count, sssp::FdCfg<LOG2L>::NT, 0, st>>>(d);
  return cudaGetLastError();
}

float4 split_ff(std::complex<double> v) {
  const float hr = float(v.real()), hi = float(v.imag());
  return make_float4(hr, hi, float(v.real() - double(hr)), float(v.imag() - double(hi)));
}

}  // namespace

bool supported(int log2L) { return log2L >= sssp::kFdMinLog2 && log2L <= sssp::kFdMaxLog2; }

cudaError_t launch_march(int log2L, const sssp::SolveDesc* d, int count, cudaStream_t st) {
  switch (log2L) {
    case 3: return launch_t<3>(d, count, st);
    case 4: return launch_t<4>(d, count, st);
    case 5: return launch_t<5>(d, count, st);
    case 6: return launch_t<6>(d, count, st);
    case 7: return launch_t<7>(d, count, st);
    case 8: return launch_t<8>(d, count, st);
    case 9: return launch_t<9>(d, count, st);
    case 10: return launch_t<10>(d, count, st);
    case 11: return launch_t<11>(d, count, st);
    case 12: return launch_t<12>(d, count, st);
  }
  return cudaErrorInvalidValue;
}

void factor_node(const double* V, int N, int L, double H, double k0, const std::complex<double>* b, int p,
                 float4* out) {
  using cd = std::complex<double>;
  const double dz = H / double(N + 1), s = 1.0 / ((k0 * dz) * (k0 * dz));
  for (int j = 0; j < p; ++j) {
    float4* tab = out + size_t(j) * L * 3;  // FdEntry = 3 float4 per point
    const cd e = b[j] * s;
    for (int q = 0; q < 3; ++q) tab[q] = make_float4(0.f, 0.f, 0.f, 0.f);  // index 0: the boundary
    cd cprev(0.0, 0.0);
    for (int n = 1; n <= N; ++n) {
      const cd dn = 1.0 + b[j] * (V[n - 1] - 2.0 * s);
      const cd den = (n == 1) ? dn : dn - e * cprev;
      const cd inv = 1.0 / den;
      const cd cp = (n < N) ? e * inv : cd(0.0, 0.0);
      float4* ent = tab + size_t(n) * 3;
      ent[0] = split_ff(inv);
      ent[1] = split_ff(-e * inv);
      ent[2] = split_ff(-cp);
      cprev = cp;
    }
  }
}

}  // namespace sssp_fd
