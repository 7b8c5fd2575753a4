// Host FP64 Pade plan (Section 2) shared by the plan builder and the C ABI.
#pragma once
#include <complex>
#include <string>

namespace sssp {

constexpr int kMaxPade = 8;

struct PadeData {
  int p = 0;
  double sigma = 0.0;
  std::complex<double> b[kMaxPade];   // Q(X) = prod_j (1 + b_j X)
  std::complex<double> a[kMaxPade];   // P(X) = prod_j (1 + a_j X), a_j = conj(b_j)
  std::complex<double> d0;            // sum form: d0 + sum_j d_j / (1 + b_j X)
  std::complex<double> d[kMaxPade];
};

// [p/p] Pade approximant of exp(i sigma (sqrt(1 + X) - 1)) at X = 0; false + message on failure.
bool pade_compute(double sigma, int p, PadeData* out, std::string* err);

}  // namespace sssp
