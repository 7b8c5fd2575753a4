// Host FP64 Pade plan for the SSSP marcher (Section 2: the [p/p] Pade approximation of the
// propagator, "computed according to Baker"; Algorithm 1's precomputation step).
//
// f(X) = exp(i sigma (sqrt(1 + X) - 1)) is expanded to order 2p, the denominator
// Q = 1 + q_1 X + .. + q_p X^p solves Baker's p x p linear system, the numerator P follows
// from the low-order Taylor products, the roots of Q give b_j (Q = prod (1 + b_j X)), and
// the residues give the sum form d0 + sum_j d_j / (1 + b_j X).  For this f the numerator is
// the complex conjugate of the denominator (checked below), so a_j = conj(b_j) and every
// product-form factor is unimodular on the real axis.
#include "pade_host.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <string>
#include <vector>

namespace sssp {

using cd = std::complex<double>;

static void taylor(double sigma, int order, std::vector<cd>& c) {
  // sqrt(1+X) - 1 = sum_{k>=1} binom(1/2, k) X^k ;  f = exp(h), h = i sigma g:
  // k f_k = sum_{j=1..k} j h_j f_{k-j}
  std::vector<double> g(order + 1, 0.0);
  if (order >= 1) g[1] = 0.5;
  for (int k = 1; k < order; ++k) g[k + 1] = g[k] * (0.5 - k) / (k + 1);
  c.assign(order + 1, cd(0, 0));
  c[0] = 1.0;
  for (int k = 1; k <= order; ++k) {
    cd s(0, 0);
    for (int j = 1; j <= k; ++j) s += double(j) * cd(0, sigma * g[j]) * c[k - j];
    c[k] = s / double(k);
  }
}

// Gaussian elimination with partial pivoting, A is n x n row-major; solves A x = rhs.
static bool solve_linear(std::vector<cd> A, std::vector<cd> rhs, int n, std::vector<cd>& x) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::abs(A[r * n + col]) > std::abs(A[piv * n + col])) piv = r;
    if (std::abs(A[piv * n + col]) == 0.0) return false;
    if (piv != col) {
      for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
      std::swap(rhs[col], rhs[piv]);
    }
    for (int r = col + 1; r < n; ++r) {
      cd f = A[r * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
      rhs[r] -= f * rhs[col];
    }
  }
  x.assign(n, cd(0, 0));
  for (int r = n - 1; r >= 0; --r) {
    cd s = rhs[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
    x[r] = s / A[r * n + r];
  }
  return true;
}

static cd polyval(const std::vector<cd>& asc, cd x) {
  cd s(0, 0);
  for (int k = int(asc.size()) - 1; k >= 0; --k) s = s * x + asc[k];
  return s;
}

// All roots of the polynomial with ascending coefficients `asc` (degree n = size-1) by
// Durand-Kerner (Weierstrass) iteration followed by Newton polishing.
static bool poly_roots(const std::vector<cd>& asc, std::vector<cd>& roots) {
  const int n = int(asc.size()) - 1;
  roots.assign(n, cd(0, 0));
  if (n == 0) return true;
  const cd lead = asc[n];
  if (std::abs(lead) == 0.0) return false;
  // Cauchy bound on the root moduli
  double bound = 0.0;
  for (int k = 0; k < n; ++k) bound = std::max(bound, std::abs(asc[k] / lead));
  bound += 1.0;
  const cd seed(0.4, 0.9);
  cd pw(1.0, 0.0);
  for (int i = 0; i < n; ++i) {
    roots[i] = bound * 0.5 * pw;
    pw *= seed;
  }
  for (int it = 0; it < 2000; ++it) {
    double change = 0.0;
    for (int i = 0; i < n; ++i) {
      cd den = lead;
      for (int j = 0; j < n; ++j)
        if (j != i) den *= (roots[i] - roots[j]);
      if (std::abs(den) == 0.0) den = cd(1e-300, 0);
      cd delta = polyval(asc, roots[i]) / den;
      roots[i] -= delta;
      change = std::max(change, std::abs(delta) / std::max(1.0, std::abs(roots[i])));
    }
    if (change < 1e-16) break;
  }
  // Newton polish on the full polynomial
  std::vector<cd> der(n);
  for (int k = 1; k <= n; ++k) der[k - 1] = double(k) * asc[k];
  for (int i = 0; i < n; ++i)
    for (int it = 0; it < 4; ++it) {
      cd dv = polyval(der, roots[i]);
      if (std::abs(dv) == 0.0) break;
      roots[i] -= polyval(asc, roots[i]) / dv;
    }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(roots[i].real()) || !std::isfinite(roots[i].imag())) return false;
  return true;
}

bool pade_compute(double sigma, int p, PadeData* out, std::string* err) {
  if (p < 1 || p > kMaxPade) {
    if (err) *err = "pade order must be in [1, 8]";
    return false;
  }
  std::vector<cd> c;
  taylor(sigma, 2 * p, c);
  // Baker: rows k = p+1..2p of (Q f - P) = 0:  sum_{i=1..p} q_i c_{k-i} = -c_k
  std::vector<cd> A(p * p), rhs(p), qv;
  for (int r = 0; r < p; ++r) {
    int k = p + 1 + r;
    for (int i = 1; i <= p; ++i) A[r * p + (i - 1)] = c[k - i];
    rhs[r] = -c[k];
  }
  if (!solve_linear(A, rhs, p, qv)) {
    if (err) *err = "Pade linear system is singular";
    return false;
  }
  std::vector<cd> q(p + 1), P(p + 1);
  q[0] = 1.0;
  for (int i = 1; i <= p; ++i) q[i] = qv[i - 1];
  for (int k = 0; k <= p; ++k) {
    cd s(0, 0);
    for (int i = 0; i <= k; ++i) s += q[i] * c[k - i];
    P[k] = s;
  }
  // the numerator must be the conjugate of the denominator (unimodular approximant)
  double qmax = 0.0, dev = 0.0;
  for (int k = 0; k <= p; ++k) {
    qmax = std::max(qmax, std::abs(q[k]));
    dev = std::max(dev, std::abs(P[k] - std::conj(q[k])));
  }
  if (!(dev <= 1e-6 * qmax)) {
    if (err) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "Pade numerator deviates from conj(denominator) by %.3g (sigma=%g, p=%d)",
                    dev / qmax, sigma, p);
      *err = buf;
    }
    return false;
  }
  std::vector<cd> xr;
  if (!poly_roots(q, xr)) {
    if (err) *err = "root finding for the Pade denominator failed";
    return false;
  }
  out->p = p;
  out->sigma = sigma;
  std::vector<cd> b(p);
  for (int j = 0; j < p; ++j) b[j] = -1.0 / xr[j];
  std::sort(b.begin(), b.end(), [](const cd& x, const cd& y) {
    return x.real() < y.real() || (x.real() == y.real() && x.imag() < y.imag());
  });
  for (int j = 0; j < p; ++j) {
    out->b[j] = b[j];
    out->a[j] = std::conj(b[j]);
  }
  out->d0 = P[p] / q[p];
  for (int j = 0; j < p; ++j) {
    cd den(1, 0);
    for (int l = 0; l < p; ++l)
      if (l != j) den *= (1.0 - b[l] / b[j]);
    out->d[j] = polyval(P, -1.0 / b[j]) / den;
  }
  return true;
}

}  // namespace sssp
