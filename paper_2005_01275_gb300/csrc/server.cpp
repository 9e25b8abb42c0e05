// Request loop for many independent solves: continuous batching over the public C ABI.
//
// Requests (each its own mesh, coefficients, data and options) are queued on submit. Up to `max_inflight` worker
// threads take them in arrival order as soon as their estimated device memory fits in the budget; each worker
// builds the request's hierarchy (nlmg_setup, host threads), solves it on the context's own CUDA stream and
// releases the memory, so requests that arrive while others run start as soon as slots and memory free up, and
// their GPU work overlaps. A request's result does not depend on what else runs: each context owns its buffers and
// every reduction has a fixed order.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nlmg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  // owned copies of the mesh and data
  int32_t n_cells = 0, n_faces = 0;
  std::vector<double> vol, ht, area, f, g;
  std::vector<int32_t> fc;
  std::vector<uint8_t> bc;
  nlmg_kappa kappa{};
  nlmg_options opt{};
  double tol_rel = 1e-8, tol_abs = 1e-10;
  int32_t max_cycles = 50;
  size_t mem_estimate = 0;
  Clock::time_point t_submit, t_start, t_setup, t_done;
  // result
  nlmg_status status = NLMG_OK;
  std::vector<double> p;
  nlmg_report rep{};
  bool done = false;
};

}  // namespace

struct nlmg_server {
  nlmg_server_options o{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  size_t mem_in_use = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
};

namespace {

// Conservative device-memory estimate of one context (fine level, CG work vectors, coarse levels, transfers).
size_t estimate_bytes(const Request& r) {
  const size_t N = (size_t)r.n_cells, F = (size_t)r.n_faces;
  return 64 * 1024 * 1024 / 64 + N * 900 + F * 120;
}

void run_request(nlmg_server* s, Request& r) {
  nlmg_mesh m{r.n_cells, r.vol.data(), r.n_faces, r.fc.data(), r.ht.data(), r.bc.data(), r.area.data()};
  nlmg_ctx* ctx = nullptr;
  r.status = nlmg_setup(&m, &r.kappa, &r.opt, &ctx);
  r.t_setup = Clock::now();
  if (r.status == NLMG_OK) {
    r.p.assign(r.n_cells, 0.0);
    r.status = nlmg_solve(ctx, r.f.data(), r.g.data(), nullptr, r.tol_rel, r.tol_abs, r.max_cycles, r.p.data(),
                          &r.rep);
  }
  nlmg_destroy(ctx);
  (void)s;
}

void worker_main(nlmg_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // strict arrival order: the head of the queue waits until its memory estimate fits
      s->cv_work.wait(lk, [&] {
        return s->stopping ||
               (!s->queue.empty() && (s->mem_in_use == 0 ||
                                      s->mem_in_use + s->queue.front()->mem_estimate <= s->o.mem_budget_bytes));
      });
      if (s->stopping && s->queue.empty()) return;
      if (s->queue.empty()) continue;
      r = s->queue.front();
      s->queue.pop_front();
      s->mem_in_use += r->mem_estimate;
      r->t_start = Clock::now();
    }
    run_request(s, *r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->mem_in_use -= r->mem_estimate;
      r->t_done = Clock::now();
      r->done = true;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

void nlmg_server_default_options(nlmg_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_inflight = 8;
  o->mem_budget_bytes = (size_t)16 << 30;
  o->setup_threads_per_request = 2;
}

nlmg_status nlmg_server_create(const nlmg_server_options* opt, nlmg_server** out) {
  if (!opt || !out || opt->max_inflight < 1 || opt->mem_budget_bytes == 0) return NLMG_EINVAL;
  nlmg_server* s = new nlmg_server();
  s->o = *opt;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return NLMG_ECUDA;
  }
  for (int i = 0; i < opt->max_inflight; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return NLMG_OK;
}

nlmg_status nlmg_server_submit(nlmg_server* s, const nlmg_mesh* mesh, const nlmg_kappa* kappa,
                               const nlmg_options* opt, const double* f_cell, const double* g_face, double tol_rel,
                               double tol_abs, int32_t max_cycles, uint64_t* ticket) {
  if (!s || !mesh || !kappa || !opt || !f_cell || !g_face || !ticket || mesh->n_cells <= 0) return NLMG_EINVAL;
  auto r = std::make_shared<Request>();
  const int N = mesh->n_cells, F = mesh->n_faces;
  r->n_cells = N;
  r->n_faces = F;
  r->vol.assign(mesh->cell_volume, mesh->cell_volume + N);
  r->fc.assign(mesh->face_cells, mesh->face_cells + 2 * (size_t)F);
  r->ht.assign(mesh->half_trans, mesh->half_trans + 2 * (size_t)F);
  r->bc.assign(mesh->face_bc, mesh->face_bc + F);
  r->area.assign(mesh->face_area, mesh->face_area + F);
  r->f.assign(f_cell, f_cell + N);
  r->g.assign(g_face, g_face + F);
  r->kappa = *kappa;
  r->opt = *opt;
  if (r->opt.setup_threads == 0) r->opt.setup_threads = s->o.setup_threads_per_request;
  r->tol_rel = tol_rel;
  r->tol_abs = tol_abs;
  r->max_cycles = max_cycles;
  r->mem_estimate = estimate_bytes(*r);
  if (r->mem_estimate > s->o.mem_budget_bytes) return NLMG_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return NLMG_OK;
}

nlmg_status nlmg_server_poll(nlmg_server* s, uint64_t ticket, int32_t wait_ms, double* p_out, nlmg_report* rep,
                             nlmg_request_times* times) {
  if (!s) return NLMG_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return NLMG_EINVAL;
    r = it->second;
    if (!r->done) {
      if (wait_ms <= 0) return NLMG_ETIMEOUT;
      if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; }))
        return NLMG_ETIMEOUT;
    }
    s->all.erase(it);
  }
  if (p_out && !r->p.empty()) std::memcpy(p_out, r->p.data(), r->p.size() * sizeof(double));
  if (rep) *rep = r->rep;
  if (times) {
    times->queue_ms = ms_between(r->t_submit, r->t_start);
    times->setup_ms = ms_between(r->t_start, r->t_setup);
    times->solve_ms = ms_between(r->t_setup, r->t_done);
    times->latency_ms = ms_between(r->t_submit, r->t_done);
  }
  return r->status;
}

void nlmg_server_destroy(nlmg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
