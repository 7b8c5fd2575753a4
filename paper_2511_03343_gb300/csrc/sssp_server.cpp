// Continuous-batching serving loop for SSSP marches (pe_server_*), written against the public
// C ABI only.
//
// Requests (one range march each: grid, Pade plan, starter, profile nodes, range) queue in
// arrival order.  At every pe_server_step the loop
//   1. admits queued requests in order while a slot is free and the plan's device bytes
//      (pe_plan_bytes_estimate) fit in what is left of the memory budget,
//   2. advances every live solve with one batched march (one kernel launch per grid size,
//      each with its own step count): the costliest kind of request live by `chunk_steps`
//      range steps, cheaper ones by proportionally more (pacing, pe_server_set_pacing),
//   3. retires the solves that reached their range: reads field and TL rows to host memory
//      and frees the plan, so the next queued requests can be admitted.
// A request that arrives while others are on the GPU joins them at the next step; all live
// solves share every launch.  Marching in chunks gives the same bits as one long march.
//
// Admission may also adapt a request so that its Neumann series (Eq. Neumann) converges:
//   PE_ADMIT_MINIMAX_C0  picks the reference sound speed c0 that minimises max|V| over the
//                        request's profile nodes (V = n^2 - 1): with n^2 = (c0/c)^2 the
//                        rescaling n^2 -> s n^2, k0 -> k0/sqrt(s), s = 2/(min n^2 + max n^2),
//                        keeps k0^2 n^2 = (omega/c)^2 and centres V on zero;
//   PE_ADMIT_CONVERGENT_ORDER chooses the Pade order from the contraction rate rho_j of the
//                        Neumann operator -b_j L_j^{-1} V (bounded in FP64 by
//                        max|V| max_m |b_j/(1 + b_j lambda_m)|; where the bound is not small
//                        enough, an FP64 power iteration with a host FFT DST-I, on the
//                        request's grid or, beyond 1023 points, on a sub-grid that resolves the
//                        modes m <= 4 k0 H/pi).  For a short step (sigma = k0 dr < 10) the
//                        order is lowered until every rho_j <= 0.3: there high orders
//                        (7 and 8 measured) leave a cut 12-term series whose march grows
//                        without bound over the range even where rho_j < 1.  Otherwise the
//                        order is lowered only while the series diverges (rho_j >= 0.98).
//                        A request that diverges at every order fails at admission.  A march
//                        that still fails on the device (a non-finite value or a diverging
//                        series reported by its status word after a chunk) is restarted from
//                        its starter one order lower, up to 8 times.
// The values used are reported by pe_server_request_params.
#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sssp.h"

namespace {

using cd = std::complex<double>;

// in-place radix-2 FFT, X_k = sum_n x_n e^{-2 pi i n k/n}, n a power of two (host FP64)
void fft_pow2(std::vector<cd>& a) {
  const size_t n = a.size();
  thread_local std::vector<cd> tw;  // e^{-2 pi i k/n}, k < n/2, for the last size used
  if (tw.size() != n / 2) {
    tw.resize(n / 2);
    for (size_t k = 0; k < n / 2; ++k) tw[k] = std::polar(1.0, -2.0 * M_PI * double(k) / double(n));
  }
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t step = n / len;
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const cd w = tw[k * step];
        const cd u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

// unnormalised DST-I of x_1..x_N (Section 3.1): S_k = sum_n x_n sin(pi n k/L), L = N + 1, from
// the DFT Z of the odd extension of length 2L (z_n = x_n, z_{2L-n} = -x_n): S_k = (i/2) Z_k
void dst1_host(const std::vector<cd>& x, std::vector<cd>& out) {
  const size_t N = x.size(), L = N + 1;
  std::vector<cd> z(2 * L, cd(0.0, 0.0));
  for (size_t n = 1; n <= N; ++n) {
    z[n] = x[n - 1];
    z[2 * L - n] = -x[n - 1];
  }
  fft_pow2(z);
  out.resize(N);
  for (size_t k = 1; k <= N; ++k) out[k - 1] = cd(0.0, 0.5) * z[k];
}

// Spectral radius estimate of M = -b L^{-1} V, L^{-1} = IDST diag(1/(1 + b lambda_m)) DST, by
// power iteration: the geometric mean growth of ||M^k x|| over iterations 16..48 (the radius
// near 1, where admission decides, is a well separated eigenvalue in the workloads; nearly
// equal moduli far below 1 converge more slowly but do not change the decision).
double neumann_radius(const std::vector<double>& V, cd b, double k0, double H) {
  const size_t N = V.size();
  const double L = double(N + 1);
  std::vector<cd> x(N), y;
  unsigned long long st = 88172645463325252ull;  // fixed xorshift start vector
  for (size_t n = 0; n < N; ++n) {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    x[n] = cd(double(st % 1000003) / 1000003.0 - 0.5, double((st >> 20) % 1000003) / 1000003.0 - 0.5);
  }
  double lg = 0.0, lg16 = 0.0;
  for (int it = 1; it <= 48; ++it) {
    double nx = 0.0;
    for (auto& v : x) nx += std::norm(v);
    nx = std::sqrt(nx);
    if (!(nx > 0.0) || !std::isfinite(nx)) return 0.0;
    for (size_t n = 0; n < N; ++n) x[n] *= V[n] / nx;
    dst1_host(x, y);
    for (size_t m = 1; m <= N; ++m) {
      const double lam = -std::pow(M_PI * double(m) / (k0 * H), 2.0);
      y[m - 1] *= (2.0 / L) / (1.0 + b * lam);
    }
    dst1_host(y, x);
    for (auto& v : x) v *= -b;
    double nn = 0.0;
    for (auto& v : x) nn += std::norm(v);
    lg += 0.5 * std::log(std::max(nn, 1e-300));
    if (it == 16) lg16 = lg;
  }
  return std::exp((lg - lg16) / 32.0);
}

struct Request {
  unsigned long long id = 0;
  int restarts = 0;        // marches restarted one Pade order lower after a device failure
  bool adapted = false;    // admission has run (a restart keeps its reference sound speed)
  pe_request r{};          // as admitted (k0, n2 and pade_order may be adapted)
  std::vector<float> u0;
  std::vector<double> n2;
  std::vector<double> node_r;
  size_t bytes = 0;
  long long tl_rows = 0;
};

struct Live {
  std::unique_ptr<Request> req;
  pe_plan* plan = nullptr;
  long long done = 0;
};

struct Result {
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  std::vector<float> field;
  std::vector<float> tl;
  long long rows = 0;
  std::string err;
  double k0 = 0.0, n2_scale = 1.0;  // the values admission marched with
  int pade_order = 0;
};

}  // namespace

struct pe_server {
  size_t budget = 0, in_use = 0, peak = 0;
  int max_live = 0, chunk = 0, peak_live = 0;
  int max_weight = 64;  // pacing: a small grid marches up to this many chunks per step
  void* stream = nullptr;
  unsigned long long next_id = 1;
  std::deque<std::unique_ptr<Request>> queue;
  std::vector<Live> live;
  std::map<unsigned long long, Result> results;
  std::string err;
};

namespace {

pe_status sfail(pe_server* s, pe_status st, const std::string& m) {
  s->err = m;
  return st;
}

long long tl_rows_for(const pe_request& r) { return r.tl_every > 0 ? r.steps / r.tl_every : 0; }

// Admission thresholds on the contraction rate rho of the Neumann series (see the file comment)
constexpr double kLowSigma = 10.0;      // sigma = k0 dr below which orders are lowered to rho <= kRhoLow
constexpr double kRhoLow = 0.3;
constexpr double kRhoConverge = 0.98;  // above: the series does not converge
constexpr int kMaxRestarts = 8;

// GPU work of one range step of a request, up to a constant: its transform count per step
// (1 + p (terms - 1) at most) times the work of one transform of L = N + 1 points (L log2 L)
double step_cost(const pe_request& r) {
  const double L = double(r.N) + 1.0;
  return L * std::log2(L) * (1.0 + double(r.pade_order) * double(std::max(r.neumann_terms - 1, 0)));
}

// Adapt a request at admission (see the file comment); false + message if it cannot converge.
bool admit_adapt(Request* q, Result* res, std::string* err) {
  pe_request& r = q->r;
  if (q->adapted) {  // a restart: the order was lowered by the restart itself
    res->pade_order = r.pade_order;
    return true;
  }
  q->adapted = true;
  res->k0 = r.k0;
  res->pade_order = r.pade_order;
  res->n2_scale = 1.0;
  if (r.neumann_terms <= 1 || r.nodes < 1) return true;
  const size_t N = size_t(r.N);
  if (r.flags & PE_ADMIT_MINIMAX_C0) {
    double lo = 1e300, hi = -1e300;
    for (double v : q->n2) {
      lo = std::min(lo, v);
      hi = std::max(hi, v);
    }
    if (lo > 0.0 && std::isfinite(hi)) {
      const double sc = 2.0 / (lo + hi);
      for (double& v : q->n2) v *= sc;
      r.k0 /= std::sqrt(sc);
      res->n2_scale = sc;
      res->k0 = r.k0;
    }
  }
  if (!(r.flags & PE_ADMIT_CONVERGENT_ORDER)) return true;
  // the node with the largest max|V| decides
  int worst = 0;
  double vmax = -1.0;
  for (int k = 0; k < r.nodes; ++k) {
    double m = 0.0;
    for (size_t n = 0; n < N; ++n) m = std::max(m, std::fabs(q->n2[size_t(k) * N + n] - 1.0));
    if (m > vmax) {
      vmax = m;
      worst = k;
    }
  }
  // the power iteration's grid: the request's, or a sub-grid (every stride-th point, N + 1 a
  // power of two) of at least 1023 points resolving the modes m <= 4 k0 H / pi
  size_t Nc = N;
  if (N > 1023) {
    const double need = 4.0 * r.k0 * r.H / M_PI;
    size_t Lc = 1024;
    while (Lc < need && Lc < N + 1) Lc *= 2;
    Nc = std::min(Lc, N + 1) - 1;
  }
  const size_t stride = (N + 1) / (Nc + 1);
  std::vector<double> V(Nc);
  for (size_t n = 0; n < Nc; ++n) V[n] = q->n2[size_t(worst) * N + (n + 1) * stride - 1] - 1.0;
  // the largest contraction rate over the Pade terms of order p (the FP64 bound where it is
  // below `enough`, else the power-iteration estimate)
  auto rate = [&](int p, double enough) {
    double b[16], a[16], d[18];
    if (pe_pade_coefficients(r.k0 * r.dr, p, b, a, d) != PE_OK) return 1e300;
    double worst_rho = 0.0;
    for (int j = 0; j < p; ++j) {
      const cd bj(b[2 * j], b[2 * j + 1]);
      double mx = 0.0;
      for (size_t m = 1; m <= N; ++m) {
        const double lam = -std::pow(M_PI * double(m) / (r.k0 * r.H), 2.0);
        mx = std::max(mx, std::abs(bj / (1.0 + bj * lam)));
      }
      const double bound = vmax * mx;
      worst_rho = std::max(worst_rho, bound <= enough ? bound : neumann_radius(V, bj, r.k0, r.H));
    }
    return worst_rho;
  };
  const double sigma = r.k0 * r.dr;
  if (sigma < kLowSigma) {
    // low frequency / short step: the highest order whose cut series contracts fast enough
    for (int p = r.pade_order; p >= 1; --p) {
      if (rate(p, kRhoLow) <= kRhoLow) {
        r.pade_order = p;
        res->pade_order = p;
        return true;
      }
    }
  }
  // otherwise the highest order at which the series converges at all
  for (int p = r.pade_order; p >= 1; --p) {
    if (rate(p, kRhoConverge) < kRhoConverge) {
      r.pade_order = p;
      res->pade_order = p;
      return true;
    }
  }
  *err = "the Neumann series diverges at every Pade order for this profile";
  return false;
}

// create the plan of a request: tables, output, profile, starter (all host -> device copies)
pe_status start_plan(pe_server* s, Request* q, pe_plan** out) {
  const pe_request& r = q->r;
  pe_plan* p = nullptr;
  pe_status st = pe_plan_create(&p, r.N, r.H, r.k0, r.dr, r.pade_order, r.neumann_terms, r.neumann_tol, s->stream);
  if (st != PE_OK) return sfail(s, st, pe_create_error());
  if ((st = pe_set_output(p, r.tl_every)) == PE_OK && r.nodes > 0)
    st = pe_set_profiles(p, q->n2.data(), q->node_r.data(), r.nodes, 0);
  if (st == PE_OK) st = pe_set_field(p, q->u0.data(), 0, r.r0);
  if (st != PE_OK) {
    s->err = pe_last_error(p);
    pe_plan_destroy(p);
    return st;
  }
  *out = p;
  return PE_OK;
}

}  // namespace

extern "C" {

pe_status pe_server_create(pe_server** out, size_t hbm_budget_bytes, int max_live, int chunk_steps, void* cuda_stream) {
  if (!out || hbm_budget_bytes == 0 || max_live < 1 || chunk_steps < 1) return PE_ERR_ARG;
  pe_server* s = new pe_server();
  s->budget = hbm_budget_bytes;
  s->max_live = max_live;
  s->chunk = chunk_steps;
  s->stream = cuda_stream;
  *out = s;
  return PE_OK;
}

pe_status pe_server_set_pacing(pe_server* s, int max_weight) {
  if (!s) return PE_ERR_ARG;
  if (max_weight < 1 || max_weight > 4096) return sfail(s, PE_ERR_ARG, "max_weight must be in [1, 4096]");
  s->max_weight = max_weight;
  return PE_OK;
}

void pe_server_destroy(pe_server* s) {
  if (!s) return;
  for (auto& l : s->live) pe_plan_destroy(l.plan);
  delete s;
}

const char* pe_server_error(const pe_server* s) { return s ? s->err.c_str() : ""; }

pe_status pe_server_submit(pe_server* s, const pe_request* r, unsigned long long* id) {
  if (!s || !r || !id) return PE_ERR_ARG;
  if (!r->u0 || r->steps < 0 || r->N < 1 || (r->neumann_terms > 1 && (r->nodes < 1 || !r->n2 || !r->node_r)))
    return sfail(s, PE_ERR_ARG, "request: missing starter or profile, or negative steps");
  auto q = std::make_unique<Request>();
  q->id = s->next_id++;
  q->r = *r;
  q->u0.assign(r->u0, r->u0 + 2 * size_t(r->N));
  if (r->nodes > 0 && r->n2) {
    q->n2.assign(r->n2, r->n2 + size_t(r->nodes) * r->N);
    q->node_r.assign(r->node_r, r->node_r + r->nodes);
  } else {
    q->r.nodes = 0;
  }
  q->r.u0 = nullptr;
  q->r.n2 = nullptr;
  q->r.node_r = nullptr;
  q->tl_rows = tl_rows_for(q->r);
  q->bytes = pe_plan_bytes_estimate(r->N, r->pade_order, q->r.nodes, q->tl_rows);
  if (q->bytes > s->budget) return sfail(s, PE_ERR_OOM, "request larger than the whole memory budget");
  *id = q->id;
  s->results[q->id].state = 0;
  s->queue.push_back(std::move(q));
  return PE_OK;
}

pe_status pe_server_step(pe_server* s, int* live_out, int* queued_out, int* completed_out) {
  if (!s) return PE_ERR_ARG;
  // 1. admission, in arrival order
  while (!s->queue.empty() && int(s->live.size()) < s->max_live && s->in_use + s->queue.front()->bytes <= s->budget) {
    std::unique_ptr<Request> q = std::move(s->queue.front());
    s->queue.pop_front();
    pe_plan* p = nullptr;
    Result& res = s->results[q->id];
    std::string aerr;
    if (!admit_adapt(q.get(), &res, &aerr)) {
      res.state = 3;
      res.err = aerr;
      continue;
    }
    pe_status st = start_plan(s, q.get(), &p);
    if (st != PE_OK) {
      res.state = 3;
      res.err = s->err;
      continue;
    }
    res.state = 1;
    s->in_use += q->bytes;
    s->peak = std::max(s->peak, s->in_use);
    Live l;
    l.req = std::move(q);
    l.plan = p;
    s->live.push_back(std::move(l));
  }
  s->peak_live = std::max(s->peak_live, int(s->live.size()));
  // 2. one batched march of every live solve.  Pacing: the grid sizes march as concurrent
  //    launches, and the step lasts as long as the slowest, so a request of the costliest kind
  //    live marches `chunk` steps and a cheaper one w chunks, w = that cost over its own (at
  //    most max_weight): small grids are not held to the pace of the largest.
  int completed = 0;
  if (!s->live.empty()) {
    std::vector<pe_plan*> plans;
    std::vector<int> steps;
    double cmax = 0.0;
    for (auto& l : s->live) cmax = std::max(cmax, step_cost(l.req->r));
    for (auto& l : s->live) {
      const double w = std::min(double(s->max_weight), std::max(1.0, std::floor(cmax / step_cost(l.req->r))));
      plans.push_back(l.plan);
      const long long n = std::min<long long>((long long)(double(s->chunk) * w), l.req->r.steps - l.done);
      steps.push_back(int(std::min<long long>(n, INT_MAX)));
    }
    pe_status st = pe_march_batch_steps(plans.data(), steps.data(), int(plans.size()));
    if (st != PE_OK) return sfail(s, st, pe_last_error(plans[0]));
    for (size_t i = 0; i < s->live.size(); ++i) s->live[i].done += steps[i];
    // 3. a march whose device status reports a failure (non-finite value, diverging series) is
    //    restarted from its starter one Pade order lower when its request allows it; then the
    //    finished solves retire (reads synchronise the stream)
    std::vector<Live> keep;
    std::vector<std::unique_ptr<Request>> again;
    for (auto& l : s->live) {
      const pe_status ds = pe_sync(l.plan);
      if (ds == PE_ERR_NUMERIC || ds == PE_ERR_NEUMANN_DIVERGED) {
        Result& res = s->results[l.req->id];
        const bool retry = (l.req->r.flags & PE_ADMIT_CONVERGENT_ORDER) && l.req->r.pade_order > 1 &&
                           l.req->restarts < kMaxRestarts;
        pe_plan_destroy(l.plan);
        s->in_use -= l.req->bytes;
        if (retry) {
          l.req->r.pade_order -= 1;
          l.req->restarts += 1;
          res.state = 0;
          again.push_back(std::move(l.req));
        } else {
          res.state = 3;
          res.err = ds == PE_ERR_NUMERIC ? "non-finite value in the march" : "Neumann series diverged";
        }
        continue;
      }
      if (l.done < l.req->r.steps) {
        keep.push_back(std::move(l));
        continue;
      }
      Result& res = s->results[l.req->id];
      res.field.resize(2 * size_t(l.req->r.N));
      pe_status rs = pe_read_field(l.plan, res.field.data(), 0);
      size_t rows = 0;
      if (rs == PE_OK) {
        res.tl.resize(size_t(l.req->tl_rows) * l.req->r.N);
        rs = pe_read_TL(l.plan, res.tl.empty() ? nullptr : res.tl.data(), res.tl.size(), nullptr, &rows);
      }
      res.rows = (long long)rows;
      res.state = (rs == PE_OK) ? 2 : 3;
      if (rs != PE_OK) res.err = pe_last_error(l.plan);
      pe_plan_destroy(l.plan);
      s->in_use -= l.req->bytes;
      ++completed;
    }
    s->live = std::move(keep);
    for (auto it = again.rbegin(); it != again.rend(); ++it) s->queue.push_front(std::move(*it));
  }
  if (live_out) *live_out = int(s->live.size());
  if (queued_out) *queued_out = int(s->queue.size());
  if (completed_out) *completed_out = completed;
  return PE_OK;
}

pe_status pe_server_state(pe_server* s, unsigned long long id, int* state) {
  if (!s || !state) return PE_ERR_ARG;
  auto it = s->results.find(id);
  if (it == s->results.end()) return sfail(s, PE_ERR_ARG, "unknown request id");
  *state = it->second.state;
  return PE_OK;
}

pe_status pe_server_take(pe_server* s, unsigned long long id, float* field, float* tl, size_t tl_cap, size_t* rows) {
  if (!s) return PE_ERR_ARG;
  auto it = s->results.find(id);
  if (it == s->results.end()) return sfail(s, PE_ERR_ARG, "unknown request id");
  Result& r = it->second;
  if (r.state == 3) {  // reported once; the entry goes so failed requests do not pile up
    const std::string m = "request failed: " + r.err;
    s->results.erase(it);
    return sfail(s, PE_ERR_CUDA, m);
  }
  if (r.state != 2) return sfail(s, PE_ERR_STATE, "request not finished");
  if (rows) *rows = size_t(r.rows);
  if (field) std::memcpy(field, r.field.data(), sizeof(float) * r.field.size());
  if (tl) {
    if (tl_cap < r.tl.size()) return sfail(s, PE_ERR_ARG, "TL buffer too small");
    std::memcpy(tl, r.tl.data(), sizeof(float) * r.tl.size());
  }
  if (field || tl) s->results.erase(it);
  return PE_OK;
}

pe_status pe_server_cancel(pe_server* s, unsigned long long id) {
  if (!s) return PE_ERR_ARG;
  auto it = s->results.find(id);
  if (it == s->results.end()) return sfail(s, PE_ERR_ARG, "unknown request id");
  if (it->second.state >= 2) return sfail(s, PE_ERR_STATE, "request already finished");
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if ((*q)->id == id) {
      s->queue.erase(q);
      break;
    }
  for (auto l = s->live.begin(); l != s->live.end(); ++l)
    if (l->req->id == id) {
      pe_sync(l->plan);  // nothing of it may still run when its memory goes
      pe_plan_destroy(l->plan);
      s->in_use -= l->req->bytes;
      s->live.erase(l);
      break;
    }
  it->second.state = 3;
  it->second.err = "cancelled";
  return PE_OK;
}

pe_status pe_neumann_radius_estimate(const double* V, int N, double H, double k0, double b_re, double b_im,
                                     double* rho) {
  if (!V || !rho || N < 1 || ((N + 1) & N) != 0 || !(H > 0) || !(k0 > 0)) return PE_ERR_ARG;
  *rho = neumann_radius(std::vector<double>(V, V + N), cd(b_re, b_im), k0, H);
  return PE_OK;
}

pe_status pe_server_request_params(pe_server* s, unsigned long long id, double* k0, double* n2_scale,
                                   int* pade_order) {
  if (!s) return PE_ERR_ARG;
  auto it = s->results.find(id);
  if (it == s->results.end()) return sfail(s, PE_ERR_ARG, "unknown request id");
  if (it->second.state == 0) return sfail(s, PE_ERR_STATE, "request not admitted yet");
  if (k0) *k0 = it->second.k0;
  if (n2_scale) *n2_scale = it->second.n2_scale;
  if (pade_order) *pade_order = it->second.pade_order;
  return PE_OK;
}

pe_status pe_server_stats(pe_server* s, size_t* bytes_in_use, size_t* peak_bytes, int* peak_live) {
  if (!s) return PE_ERR_ARG;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (peak_bytes) *peak_bytes = s->peak;
  if (peak_live) *peak_live = s->peak_live;
  return PE_OK;
}

}  // extern "C"
