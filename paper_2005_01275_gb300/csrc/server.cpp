// Request loop for many independent solves: continuous batching over the public C ABI.
//
// Requests (each its own mesh, coefficients, data and options) are queued on submit. Up to `max_inflight` worker
// threads take them in arrival order as soon as their estimated device memory fits in the budget; each worker
// builds the request's hierarchy (nlmg_setup) or, when an identical mesh with identical hierarchy options was seen
// before and its hierarchy is still kept, makes an nlmg_instance of it; it solves on the context's own CUDA stream and
// releases the work memory, so requests that arrive while others run start as soon as slots and memory free up, and
// their GPU work overlaps. A request's result does not depend on what else runs or on reuse: each context owns its
// work buffers, every reduction has a fixed order and the setup is deterministic.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
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
  uint64_t key = 0;   // hash of the mesh arrays and hierarchy options
  int reused = 0;
  Clock::time_point t_submit, t_start, t_setup, t_done;
  // result
  nlmg_status status = NLMG_OK;
  std::vector<double> p;
  nlmg_report rep{};
  bool done = false;
};

// A hierarchy kept on the device after its request: the context that built it, and what identifies it.
struct Kept {
  uint64_t key = 0;
  std::shared_ptr<Request> like;   // the request that built it (its mesh arrays and options)
  nlmg_ctx* base = nullptr;
  size_t bytes = 0;
  uint64_t last_used = 0;
  int in_use = 0;
};

}  // namespace

struct nlmg_server {
  nlmg_server_options o{};
  int device = 0;
  int sms = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  size_t mem_in_use = 0;
  std::list<std::shared_ptr<Kept>> kept;
  size_t kept_bytes = 0;
  uint64_t tick = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
};

namespace {

// Conservative device-memory estimate of one context (fine level, Krylov work vectors including the Newton and
// GMRES buffers, coarse levels, transfers); checked against the bytes contexts really hold by the GPU tests.
size_t estimate_cells_faces(size_t N, size_t F) { return ((size_t)4 << 20) + N * 2000 + F * 200; }
size_t estimate_bytes(const Request& r) { return estimate_cells_faces((size_t)r.n_cells, (size_t)r.n_faces); }

// FNV-1a over the bytes that determine a hierarchy.
struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  }
  template <class T>
  void vec(const std::vector<T>& v) {
    add(v.data(), v.size() * sizeof(T));
  }
};

uint64_t hierarchy_key(const Request& r) {
  Fnv f;
  f.add(&r.n_cells, sizeof(r.n_cells));
  f.add(&r.n_faces, sizeof(r.n_faces));
  f.vec(r.vol);
  f.vec(r.fc);
  f.vec(r.ht);
  f.vec(r.bc);
  f.vec(r.area);
  const int nl = r.opt.n_levels;
  f.add(&nl, sizeof(nl));
  for (int l = 0; l + 1 < nl; ++l) {
    f.add(&r.opt.agg_size[l], sizeof(int32_t));
    f.add(&r.opt.modes[l], sizeof(int32_t));
    f.add(&r.opt.flux_modes[l], sizeof(int32_t));
  }
  return f.h;
}

bool same_hierarchy(const Request& a, const Request& b) {
  if (a.key != b.key || a.n_cells != b.n_cells || a.n_faces != b.n_faces || a.opt.n_levels != b.opt.n_levels)
    return false;
  for (int l = 0; l + 1 < a.opt.n_levels; ++l)
    if (a.opt.agg_size[l] != b.opt.agg_size[l] || a.opt.modes[l] != b.opt.modes[l] ||
        a.opt.flux_modes[l] != b.opt.flux_modes[l])
      return false;
  return a.vol == b.vol && a.fc == b.fc && a.ht == b.ht && a.bc == b.bc && a.area == b.area;
}

// caller holds s->mu
std::shared_ptr<Kept> find_kept(nlmg_server* s, const Request& r) {
  for (auto& k : s->kept)
    if (same_hierarchy(*k->like, r)) return k;
  return nullptr;
}

// Evicts the least recently used idle kept hierarchy; caller holds s->mu. Returns false if none is idle.
bool evict_one(nlmg_server* s) {
  auto victim = s->kept.end();
  for (auto it = s->kept.begin(); it != s->kept.end(); ++it)
    if ((*it)->in_use == 0 && (victim == s->kept.end() || (*it)->last_used < (*victim)->last_used)) victim = it;
  if (victim == s->kept.end()) return false;
  nlmg_destroy((*victim)->base);
  s->kept_bytes -= (*victim)->bytes;
  s->kept.erase(victim);
  return true;
}

void solve_on(Request& r, nlmg_ctx* ctx) {
  r.p.assign(r.n_cells, 0.0);
  r.status = nlmg_solve(ctx, r.f.data(), r.g.data(), nullptr, r.tol_rel, r.tol_abs, r.max_cycles, r.p.data(), &r.rep);
}

void run_request(nlmg_server* s, const std::shared_ptr<Request>& rp, const std::shared_ptr<Kept>& hit) {
  Request& r = *rp;
  if (hit) {
    nlmg_ctx* ctx = nullptr;
    r.status = nlmg_instance(hit->base, &r.kappa, &ctx);
    if (r.status == NLMG_OK) r.status = nlmg_set_options(ctx, &r.opt);
    r.reused = 1;
    r.t_setup = Clock::now();
    if (r.status == NLMG_OK) solve_on(r, ctx);
    nlmg_destroy(ctx);
    std::lock_guard<std::mutex> lk(s->mu);
    hit->in_use--;
    return;
  }
  nlmg_mesh m{r.n_cells, r.vol.data(), r.n_faces, r.fc.data(), r.ht.data(), r.bc.data(), r.area.data()};
  nlmg_ctx* ctx = nullptr;
  r.status = nlmg_setup(&m, &r.kappa, &r.opt, &ctx);
  r.t_setup = Clock::now();
  if (r.status != NLMG_OK) {
    nlmg_destroy(ctx);
    return;
  }
  solve_on(r, ctx);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->o.hierarchy_cache <= 0 || find_kept(s, r)) {
    nlmg_destroy(ctx);
    return;
  }
  auto k = std::make_shared<Kept>();
  k->key = r.key;
  k->like = rp;
  k->base = ctx;
  k->bytes = r.mem_estimate;
  k->last_used = ++s->tick;
  s->kept.push_back(k);
  s->kept_bytes += k->bytes;
  while ((int)s->kept.size() > s->o.hierarchy_cache && evict_one(s)) {
  }
}

void worker_main(nlmg_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::shared_ptr<Request> r;
    std::shared_ptr<Kept> hit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // strict arrival order: the head of the queue waits until its memory estimate fits (kept hierarchies that
      // are idle are evicted, least recently used first, to make room)
      for (;;) {
        if (s->stopping && s->queue.empty()) return;
        if (!s->queue.empty()) {
          const size_t need = s->queue.front()->mem_estimate;
          while (s->mem_in_use + s->kept_bytes + need > s->o.mem_budget_bytes && evict_one(s)) {
          }
          if (s->mem_in_use == 0 || s->mem_in_use + s->kept_bytes + need <= s->o.mem_budget_bytes) break;
        }
        s->cv_work.wait(lk);
      }
      r = s->queue.front();
      s->queue.pop_front();
      s->mem_in_use += r->mem_estimate;
      r->t_start = Clock::now();
      hit = find_kept(s, *r);
      if (hit) {
        hit->in_use++;
        hit->last_used = ++s->tick;
      }
    }
    run_request(s, r, hit);
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

nlmg_status nlmg_server_request_bytes(const nlmg_mesh* mesh, size_t* bytes) {
  if (!mesh || !bytes || mesh->n_cells < 1 || mesh->n_faces < 0) return NLMG_EINVAL;
  *bytes = estimate_cells_faces((size_t)mesh->n_cells, (size_t)mesh->n_faces);
  return NLMG_OK;
}

void nlmg_server_default_options(nlmg_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_inflight = 8;
  o->mem_budget_bytes = (size_t)16 << 30;
  o->setup_threads_per_request = 2;
  o->hierarchy_cache = 8;
}

nlmg_status nlmg_server_create(const nlmg_server_options* opt, nlmg_server** out) {
  if (!opt || !out || opt->max_inflight < 1 || opt->mem_budget_bytes == 0) return NLMG_EINVAL;
  nlmg_server* s = new nlmg_server();
  s->o = *opt;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
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
  // requests run side by side: unless the request says otherwise, its persistent kernels use a share of the SMs
  if (r->opt.max_sms == 0 && s->o.max_inflight > 1) r->opt.max_sms = std::max(1, s->sms / std::min(s->o.max_inflight, 4));
  r->tol_rel = tol_rel;
  r->tol_abs = tol_abs;
  r->max_cycles = max_cycles;
  r->mem_estimate = estimate_bytes(*r);
  r->key = hierarchy_key(*r);
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
      // the wait released the lock: another poll of the same ticket may have released it meanwhile
      it = s->all.find(ticket);
      if (it == s->all.end() || it->second != r) return NLMG_EINVAL;
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
    times->hierarchy_reused = r->reused;
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
  for (auto& k : s->kept) nlmg_destroy(k->base);
  delete s;
}

}  // extern "C"
