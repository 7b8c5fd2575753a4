// Continuous-batching serving loop for SSSP marches (pe_server_*), written against the public
// C ABI only.
//
// Requests (one range march each: grid, Pade plan, starter, profile nodes, range) queue in
// arrival order.  At every pe_server_step the loop
//   1. admits queued requests in order while a slot is free and the plan's device bytes
//      (pe_plan_bytes_estimate) fit in what is left of the memory budget,
//   2. advances every live solve by up to `chunk_steps` range steps with one batched march
//      (one kernel launch per grid size, one CTA per solve, each with its own step count),
//   3. retires the solves that reached their range: reads field and TL rows to host memory
//      and frees the plan, so the next queued requests can be admitted.
// A request that arrives while others are on the GPU joins them at the next step; all live
// solves share every launch.  Marching in chunks gives the same bits as one long march.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sssp.h"

namespace {

struct Request {
  unsigned long long id = 0;
  pe_request r{};
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
};

}  // namespace

struct pe_server {
  size_t budget = 0, in_use = 0, peak = 0;
  int max_live = 0, chunk = 0, peak_live = 0;
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
    pe_status st = start_plan(s, q.get(), &p);
    Result& res = s->results[q->id];
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
  // 2. one batched march of every live solve
  int completed = 0;
  if (!s->live.empty()) {
    std::vector<pe_plan*> plans;
    std::vector<int> steps;
    for (auto& l : s->live) {
      plans.push_back(l.plan);
      steps.push_back(int(std::min<long long>(s->chunk, l.req->r.steps - l.done)));
    }
    pe_status st = pe_march_batch_steps(plans.data(), steps.data(), int(plans.size()));
    if (st != PE_OK) return sfail(s, st, pe_last_error(plans[0]));
    for (size_t i = 0; i < s->live.size(); ++i) s->live[i].done += steps[i];
    // 3. retire finished solves (reads synchronise the stream)
    std::vector<Live> keep;
    for (auto& l : s->live) {
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
  if (r.state == 3) return sfail(s, PE_ERR_CUDA, "request failed: " + r.err);
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

pe_status pe_server_stats(pe_server* s, size_t* bytes_in_use, size_t* peak_bytes, int* peak_live) {
  if (!s) return PE_ERR_ARG;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (peak_bytes) *peak_bytes = s->peak;
  if (peak_live) *peak_live = s->peak_live;
  return PE_OK;
}

}  // extern "C"
