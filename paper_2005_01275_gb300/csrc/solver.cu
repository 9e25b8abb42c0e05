// nlmg: context, device upload of the hierarchy, FAS cycle (Algorithm 2), backtracking (Algorithm 1), Picard
// smoothing steps, and the C ABI of include/nlmg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/nlmg.h"
#include "dense.hpp"
#include "hier.hpp"
#include "kernels.cuh"
#include "eig.cuh"
#include "mg.cuh"
#include "noalloc.cuh"
#include "persist.cuh"

using namespace nlmg;

namespace {

struct Error : std::runtime_error {
  nlmg_status code;
  Error(nlmg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                                         \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      throw Error(e_ == cudaErrorMemoryAllocation ? NLMG_ENOMEM : NLMG_ECUDA,                            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                   \
  } while (0)

// Per coarse level work buffers.
struct CoarseBuf {
  double *x = nullptr, *b = nullptr, *r = nullptr, *dx = nullptr, *nb = nullptr, *xt2 = nullptr;
  double *xc = nullptr, *yl = nullptr, *kapc = nullptr, *ptmp = nullptr;
  double *ylam = nullptr, *ydiag = nullptr, *lam = nullptr, *lr = nullptr, *lz = nullptr, *lpa = nullptr, *lpb = nullptr,
         *lq = nullptr, *ldinv = nullptr, *xi = nullptr;
  double *hw = nullptr, *hz = nullptr, *hs = nullptr, *hma = nullptr, *hmb = nullptr;   // pipelined hybridized CG
  double* hsv = nullptr;    // values of the SELL form of H
  LinParts base{}, dir{};   // linear parts of the operator at x and along dx (fused coarse step)
  double rn = 0.0;  // ||A(x) - b|| at the current x (valid after coarse_res)
};

// Optional CUDA-event timing of selected kernels on the context stream (pairs of events around each launch).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kid;
  int used = 0;
  double ms[8] = {0};
  long long n[8] = {0};
  double bytes[8] = {0};
  double flops[8] = {0};
};

// Fine-level state: iterate, its kappa and residual.
struct FineState {
  double *p = nullptr, *kap = nullptr, *R = nullptr;
  double rn = 0.0;
};

// What every instance of one setup shares: the fine mesh and the hierarchy on the host, and their read-only device
// copies (mesh arrays, level operators, transfers). Freed with the last context that refers to it.
struct Shared {
  FineMesh fm;
  Hierarchy H;
  std::vector<void*> allocs;
  size_t bytes = 0;   // device bytes of allocs
  FineDev F;
  std::vector<LevelDev> LD;
  std::vector<TransferDev> TD;
  long long nnz_real = 0;
  double hyb_bytes_per_iter[8] = {0}, hyb_bytes_per_iter_sell[8] = {0};
  double coarse_res_bytes[8] = {0};   // algorithmic bytes of one coarse operator evaluation per level
  // algorithmic flops (FMA = 2) per level: one hybridized CG iteration, the fixed work of one hybridized solve
  // (right-hand side per interface slot, local recovery), one coarse operator evaluation
  double hyb_flops_per_iter[8] = {0}, hyb_flops_per_solve[8] = {0}, coarse_res_flops[8] = {0};
  // one trial evaluation from the linear parts (also the pass that accepts a trial): bytes and flops
  double coarse_trial_bytes[8] = {0}, coarse_trial_flops[8] = {0};
  int n_fas = 0;        // levels the FAS cycles use (the hierarchy may hold more for the preconditioner)
  MgDev MG;             // multigrid preconditioner structure (MG.L = 0: not built)
  double mg_bytes_setup = 0, mg_bytes_vcycle = 0, mg_bytes_iter = 0;   // algorithmic bytes (see mg_accounting)
  ~Shared() {
    for (void* p : allocs) cudaFree(p);
  }
};

}  // namespace

struct nlmg_ctx {
  std::string err;
  nlmg_options opt{};
  int kind = 0;
  double a = 0.0;
  std::shared_ptr<Shared> sh = std::make_shared<Shared>();
  FineMesh& fm() { return sh->fm; }
  Hierarchy& H() { return sh->H; }
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;   // this context's work buffers
  size_t own_bytes = 0;        // device bytes of allocs
  FineDev F;                   // copies of the shared descriptors (device pointers into sh)
  std::vector<LevelDev> LD;
  std::vector<TransferDev> TD;
  std::vector<CoarseBuf> CB;
  int sm_cap = 0;                 // SMs the persistent kernels may use (0 = all; set while instances share the GPU)
  std::vector<nlmg_ctx*> pool;   // extra instances for multi-right-hand-side solves, created on demand
  std::mutex pool_mu;
  double* d_partial = nullptr;
  unsigned* d_cnt = nullptr;
  double* d_sc = nullptr;
  double* h_sc = nullptr;   // pinned
  // fine buffers
  double *f = nullptr, *g = nullptr, *rhs = nullptr, *dkap = nullptr, *Tval = nullptr, *dinv = nullptr,
         *diagT = nullptr, *jdiag = nullptr, *sig0 = nullptr, *ptr_e = nullptr, *fdp = nullptr;
  double *cx = nullptr, *cr = nullptr, *cz = nullptr, *cpa = nullptr, *cpb = nullptr, *cq = nullptr;
  double *sdiag = nullptr, *Ts64 = nullptr, *dv1 = nullptr, *dv2 = nullptr;
  // Newton baseline: Jacobian off-diagonals, Jacobi scaling, GMRES(30) basis and work vectors
  static constexpr int kGmresM = 30;
  double *Joff = nullptr, *jdinv = nullptr, *gV = nullptr, *gw = nullptr, *gu = nullptr, *gr = nullptr,
         *gh = nullptr, *h_gh = nullptr;
  // Newton smoothing steps: the scaled Jacobian of the BiCGStab (off-diagonal, diagonal, S); its 7 work vectors
  // are the first 7 of the GMRES basis
  double *Js = nullptr, *jdS = nullptr, *jsS = nullptr;
  float *Ts32 = nullptr, *fy = nullptr, *fr = nullptr, *fpa = nullptr, *fpb = nullptr, *fq = nullptr, *fs = nullptr;
  FineState cur, t1, t2;
  bool have_data = false;
  double tol_rel = 1e-8, tol_abs = 1e-10;   // outer tolerances, also used on the coarsest level
  double lin_tol_eff = 1e-2, coarse_lin_tol_eff = 1e-1, coarsest_lin_tol_eff = 2e-1, newton_tol_eff = 1e-2;   // inner
  // tolerances of the running solve
  int tightenings = 0;
  double r0_ref = 0.0;             // ||R(p_0)|| of the running solve (the Picard-then-Newton switch)
  bool newton_off = false;         // a Newton smoothing step of the running solve failed to halve the residual
  long long newton_steps = 0;      // level-0 Newton smoothing steps of the running solve
  int last_fine_kind = 0;          // variant of the last level-0 CG launch (0 two-barrier, 1 pipelined, 2 registers)
  int auto_sm_cap = 0;            // SM share chosen by nlmg_solve_many while instances run side by side
  void reset_inner_tols() {
    sm_cap = opt.max_sms > 0 ? opt.max_sms : auto_sm_cap;
    lin_tol_eff = opt.lin_tol;
    coarse_lin_tol_eff = opt.coarse_lin_tol;
    coarsest_lin_tol_eff = opt.coarsest_lin_tol > 0.0 ? opt.coarsest_lin_tol : opt.coarse_lin_tol;
    newton_tol_eff = opt.newton_lin_tol;
    tightenings = 0;
  }
  // statistics of the running solve
  long long fine_evals = 0, lin_iters = 0;
  long long lin_iters_level[8] = {0};
  Prof prof;
  PcgResult* d_res = nullptr;   // device result of the persistent CG kernels
  PcgResult* h_res = nullptr;   // pinned copy
  unsigned* d_bar = nullptr;    // grid barrier count / generation
  int prof_begin(int k) {
    if (!prof.on) return -1;
    if (prof.used * 2 + 2 > (int)prof.ev.size()) prof_flush();
    int i = prof.used++;
    prof.kid[i] = k;
    CK(cudaEventRecord(prof.ev[2 * i], st));
    return i;
  }
  void prof_end(int i) {
    if (i >= 0) CK(cudaEventRecord(prof.ev[2 * i + 1], st));
  }
  void prof_flush() {
    if (prof.used == 0) return;
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < prof.used; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, prof.ev[2 * i], prof.ev[2 * i + 1]));
      prof.ms[prof.kid[i]] += ms;
      prof.n[prof.kid[i]] += 1;
    }
    prof.used = 0;
  }

  // device arrays are allocated in whole 16-byte units (kernels may copy them in 16-byte chunks)
  static size_t whole16(size_t bytes) { return (std::max<size_t>(bytes, 1) + 15) & ~(size_t)15; }
  template <class T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    const size_t bytes = whole16(n * sizeof(T));
    CK(cudaMalloc(&p, bytes));
    allocs.push_back(p);
    own_bytes += bytes;
    return (T*)p;
  }
  // read-only data of the hierarchy: owned by the shared part
  template <class T>
  T* upload(const std::vector<T>& v) {
    void* p = nullptr;
    const size_t bytes = whole16(v.size() * sizeof(T));
    CK(cudaMalloc(&p, bytes));
    sh->allocs.push_back(p);
    sh->bytes += bytes;
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return (T*)p;
  }
  Reduce red(int slot) { return Reduce{d_partial, d_cnt, d_sc + slot}; }
  double read_sc(int slot) {
    CK(cudaMemcpyAsync(h_sc, d_sc + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return *h_sc;
  }
  void read_sc2(int s0, double& v0, double& v1) {  // two consecutive slots
    CK(cudaMemcpyAsync(h_sc, d_sc + s0, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    v0 = h_sc[0];
    v1 = h_sc[1];
  }
  int nlev() const { return sh->n_fas; }
  MgWork mg;               // multigrid preconditioner work buffers and graphs (when sh->MG.L > 0)
};

namespace {

// ---------------------------------------------------------------------------------------------------------------
// upload

void upload_fine(nlmg_ctx* c) {
  const FineMesh& fm = c->fm();
  const int N = fm.n_cells;
  std::vector<std::vector<int>> rows(N);
  std::vector<int> off(N + 1, 0), nbr, doff(N + 1, 0), dface, noff(N + 1, 0), nface;
  std::vector<double> us, un, dups, narea;
  std::vector<std::vector<int>> dl(N), nl(N);
  for (int f = 0; f < fm.n_faces; ++f) {
    if (fm.bc[f] == 0) {
      rows[fm.fk[f]].push_back(f);
      rows[fm.fl[f]].push_back(f);
    } else if (fm.bc[f] == 1) {
      dl[fm.fk[f]].push_back(f);
    } else {
      nl[fm.fk[f]].push_back(f);
    }
  }
  for (int K = 0; K < N; ++K) {
    for (int f : rows[K]) {
      bool own = fm.fk[f] == K;
      nbr.push_back(own ? fm.fl[f] : fm.fk[f]);
      us.push_back(own ? fm.ups0[f] : fm.ups1[f]);
      un.push_back(own ? fm.ups1[f] : fm.ups0[f]);
    }
    off[K + 1] = (int)nbr.size();
    for (int f : dl[K]) { dface.push_back(f); dups.push_back(fm.ups0[f]); }
    doff[K + 1] = (int)dface.size();
    for (int f : nl[K]) { nface.push_back(f); narea.push_back(fm.area[f]); }
    noff[K + 1] = (int)nface.size();
  }
  FineDev& F = c->F;
  F.N = N;
  F.nslice = (N + 31) / 32;
  std::vector<int> soff(F.nslice + 1, 0), sw(F.nslice, 0);
  for (int sl = 0; sl < F.nslice; ++sl) {
    int w = 0;
    for (int K = 32 * sl; K < std::min(N, 32 * sl + 32); ++K) w = std::max(w, off[K + 1] - off[K]);
    sw[sl] = w;
    soff[sl + 1] = soff[sl] + 32 * w;
  }
  std::vector<int> snbr(soff[F.nslice], 0);
  std::vector<double> sus(soff[F.nslice], 1.0), sun(soff[F.nslice], 0.0);
  for (int K = 0; K < N; ++K) {
    int sl = K >> 5, lane = K & 31, deg = off[K + 1] - off[K];
    for (int j = 0; j < sw[sl]; ++j) {
      int e = soff[sl] + 32 * j + lane;
      if (j < deg) {
        snbr[e] = nbr[off[K] + j];
        sus[e] = us[off[K] + j];
        sun[e] = un[off[K] + j];
      } else {
        snbr[e] = K;   // padding: Ups = (1, 0) gives a zero transmissibility
      }
    }
  }
  F.nnz = soff[F.nslice];
  c->sh->nnz_real = (long long)nbr.size();
  F.sell_off = c->upload(soff);
  F.sell_w = c->upload(sw);
  F.nbr = c->upload(snbr);
  F.ups_s = c->upload(sus);
  F.ups_n = c->upload(sun);
  F.dir_off = c->upload(doff);
  F.dir_face = c->upload(dface);
  F.dir_ups = c->upload(dups);
  F.neu_off = c->upload(noff);
  F.neu_face = c->upload(nface);
  F.neu_area = c->upload(narea);
  F.vol = c->upload(fm.vol);
  const Level& L0 = c->H().levels[0];
  std::vector<int> flk, fll, flf;
  std::vector<double> u0, u1;
  for (int j = 0; j < L0.n_flux; ++j) {
    int f = L0.face_of_flux[j];
    flk.push_back(fm.fk[f]);
    fll.push_back(fm.bc[f] == 0 ? fm.fl[f] : -1);
    flf.push_back(f);
    u0.push_back(fm.ups0[f]);
    u1.push_back(fm.bc[f] == 0 ? fm.ups1[f] : 0.0);
  }
  F.nflux = L0.n_flux;
  F.fl_k = c->upload(flk);
  F.fl_l = c->upload(fll);
  F.fl_face = c->upload(flf);
  F.fl_u0 = c->upload(u0);
  F.fl_u1 = c->upload(u1);
}

void upload_level(nlmg_ctx* c, int l) {
  const Level& L = c->H().levels[l];
  LevelDev& D = c->LD[l];
  D.nc = L.n_cells;
  D.nflux = L.n_flux;
  D.np = L.n_p();
  D.nyl = (int)L.loc.size();
  for (int cc = 0; cc < L.n_cells; ++cc) {
    if (L.nloc(cc) > kMaxLoc) throw Error(NLMG_EUNSUPPORTED, "a coarse cell has more than 128 flux unknowns");
    if (L.m[cc] > kMaxM) throw Error(NLMG_EUNSUPPORTED, "more than 8 modes per aggregate");
  }
  D.m = c->upload(L.m);
  D.p_off = c->upload(L.p_off);
  D.loc_off = c->upload(L.loc_off);
  D.loc = c->upload(L.loc);
  D.mat_off = c->upload(L.mat_off);
  D.dmat_off = c->upload(L.dmat_off);
  D.Mloc = c->upload(L.Mloc);
  D.Dloc = c->upload(L.Dloc);
  D.w = c->upload(L.w);
  std::vector<int> fy0(L.n_flux, -1), fy1(L.n_flux, -1), own0(L.loc.size(), 0);
  for (int cc = 0; cc < L.n_cells; ++cc)
    for (int k = L.loc_off[cc]; k < L.loc_off[cc + 1]; ++k) {
      int i = L.loc[k];
      if (L.fown0[i] == cc) { fy0[i] = k; own0[k] = 1; } else { fy1[i] = k; }
    }
  D.f_y0 = c->upload(fy0);
  D.f_y1 = c->upload(fy1);
  D.own0 = c->upload(own0);
  // hybridization data
  std::vector<int> lam_of(L.n_flux, -1);
  int nlam = 0;
  for (int i = 0; i < L.n_flux; ++i)
    if (L.fkind[i] == KIND_IFACE) lam_of[i] = nlam++;
  D.nlam = nlam;
  std::vector<int> sad_off(L.n_cells + 1, 0), if_off(L.n_cells + 1, 0), if_slot, if_lam, hc_off(L.n_cells + 1, 0);
  std::vector<double> Sinv, if_sign, Hc;
  std::vector<int> ly0(nlam, -1), ly1(nlam, -1);
  for (int cc = 0; cc < L.n_cells; ++cc) {
    int nl = L.nloc(cc), mc = L.m[cc], n = nl + mc;
    std::vector<double> K((size_t)n * n, 0.0), Ki((size_t)n * n, 0.0);
    for (int s = 0; s < nl; ++s)
      for (int t = 0; t < nl; ++t) K[(size_t)s * n + t] = L.Mloc[L.mat_off[cc] + (size_t)s * nl + t];
    for (int r = 0; r < mc; ++r)
      for (int s = 0; s < nl; ++s) {
        double d = L.Dloc[L.dmat_off[cc] + (size_t)r * nl + s];
        K[(size_t)(nl + r) * n + s] = d;
        K[(size_t)s * n + nl + r] = d;
      }
    if (!invert(n, K.data(), Ki.data())) throw Error(NLMG_EINVAL, "singular local saddle on a coarse cell");
    sad_off[cc + 1] = sad_off[cc] + n * n;
    Sinv.insert(Sinv.end(), Ki.begin(), Ki.end());
    std::vector<int> slots;
    for (int s = 0; s < nl; ++s) {
      int i = L.loc[L.loc_off[cc] + s];
      if (lam_of[i] < 0) continue;
      int k = (int)if_slot.size();
      slots.push_back(s);
      if_slot.push_back(s);
      if_lam.push_back(lam_of[i]);
      bool first = L.fown0[i] == cc;
      if_sign.push_back(first ? 1.0 : -1.0);
      (first ? ly0 : ly1)[lam_of[i]] = k;
    }
    if_off[cc + 1] = (int)if_slot.size();
    int ni = (int)slots.size();
    hc_off[cc + 1] = hc_off[cc] + ni * ni;
    for (int k = 0; k < ni; ++k)
      for (int j = 0; j < ni; ++j)
        Hc.push_back(if_sign[if_off[cc] + k] * if_sign[if_off[cc] + j] * Ki[(size_t)slots[k] * n + slots[j]]);
  }
  D.nif = (int)if_slot.size();
  D.sad_off = c->upload(sad_off);
  D.Sinv = c->upload(Sinv);
  D.if_off = c->upload(if_off);
  D.if_slot = c->upload(if_slot);
  D.if_lam = c->upload(if_lam);
  D.if_sign = c->upload(if_sign);
  D.hc_off = c->upload(hc_off);
  D.Hc = c->upload(Hc);
  D.lam_y0 = c->upload(ly0);
  D.lam_y1 = c->upload(ly1);
  std::vector<int> ifc(if_slot.size()), slc(L.loc.size()), pc(L.n_p());
  for (int cc = 0; cc < L.n_cells; ++cc) {
    for (int k = if_off[cc]; k < if_off[cc + 1]; ++k) ifc[k] = cc;
    for (int k = L.loc_off[cc]; k < L.loc_off[cc + 1]; ++k) slc[k] = cc;
    for (int k = L.p_off[cc]; k < L.p_off[cc + 1]; ++k) pc[k] = cc;
  }
  D.if_cell = c->upload(ifc);
  D.slot_cell = c->upload(slc);
  D.p_cell = c->upload(pc);
  // H as a SELL-32 matrix over the lambdas: row l takes the Hc row of each of its two slots k (cell c_k, columns the
  // lambdas of c_k's interface slots); a column met from both slots (l itself, or another lambda of the same
  // interface) gets both contributions
  {
    const int nsl = (nlam + 31) / 32;
    std::vector<int> lc0(nlam), lc1(nlam), rlen(nlam, 0), roff(nlam + 1, 0);
    std::vector<int> rcol, ri0, ri1;
    rcol.reserve((size_t)nlam * 28);
    ri0.reserve((size_t)nlam * 28);
    ri1.reserve((size_t)nlam * 28);
    for (int l = 0; l < nlam; ++l) {
      const size_t start = rcol.size();
      for (int side = 0; side < 2; ++side) {
        const int k = side == 0 ? ly0[l] : ly1[l];
        if (k < 0) throw Error(NLMG_EINVAL, "a coarse interface unknown without two cells");
        const int cc = ifc[k], k0 = if_off[cc], ni = if_off[cc + 1] - k0;
        (side == 0 ? lc0 : lc1)[l] = cc;
        for (int j = 0; j < ni; ++j) {
          const int m = if_lam[k0 + j], idx = hc_off[cc] + (k - k0) * ni + j;
          size_t q = start;
          while (q < rcol.size() && rcol[q] != m) ++q;
          if (q == rcol.size()) {
            rcol.push_back(m);
            ri0.push_back(-1);
            ri1.push_back(-1);
          }
          (side == 0 ? ri0 : ri1)[q] = idx;
        }
      }
      rlen[l] = (int)(rcol.size() - start);
      roff[l + 1] = (int)rcol.size();
    }
    std::vector<int> hw(nsl, 0), hoff(nsl + 1, 0);
    for (int s = 0; s < nsl; ++s) {
      int w = 0;
      for (int l = 32 * s; l < std::min(nlam, 32 * s + 32); ++l) w = std::max(w, rlen[l]);
      hw[s] = w;
      hoff[s + 1] = hoff[s] + 32 * w;
    }
    const int E = nsl ? hoff[nsl] : 0;
    std::vector<int> hcol(E), hi0(E, -1), hi1(E, -1);
    for (int s = 0; s < nsl; ++s)
      for (int lane = 0; lane < 32; ++lane) {
        const int l = 32 * s + lane;
        for (int j = 0; j < hw[s]; ++j) {
          const int e = hoff[s] + lane + 32 * j;
          if (l < nlam && j < rlen[l]) {
            hcol[e] = rcol[roff[l] + j];
            hi0[e] = ri0[roff[l] + j];
            hi1[e] = ri1[roff[l] + j];
          } else {
            hcol[e] = l < nlam ? l : 0;   // padding: no contribution
          }
        }
      }
    D.hs_n = E;
    D.hs_w = c->upload(hw);
    D.hs_off = c->upload(hoff);
    D.hs_col = c->upload(hcol);
    D.hs_i0 = c->upload(hi0);
    D.hs_i1 = c->upload(hi1);
    D.lam_c0 = c->upload(lc0);
    D.lam_c1 = c->upload(lc1);
    // one CG iteration on the SELL form: entries (value, column) and the gathered vector, plus the lambda vectors
    c->sh->hyb_bytes_per_iter_sell[l] = 20.0 * E + 136.0 * nlam;
  }
  // algorithmic bytes of one CG iteration of the hybridized solve: H blocks, their lambda ids, the per-interface
  // buffer written and read, the lambda vectors (z, p_old gathered once; CG update 5 reads + 3 writes)
  c->sh->hyb_bytes_per_iter[l] = 8.0 * (double)Hc.size() + 12.0 * D.nif + 8.0 * D.nc + 16.0 * D.nif + 136.0 * nlam;
  // one evaluation of the coarse operator: the static local blocks and their index arrays, x read, kappa per cell
  // written and read, the per-cell products written and read, r written
  c->sh->coarse_res_bytes[l] = 8.0 * (double)(L.Mloc.size() + L.Dloc.size()) + 8.0 * (double)L.loc.size() +
                               16.0 * (D.nflux + D.np) + 16.0 * D.nc + 16.0 * D.nyl + 8.0 * (D.nflux + D.np);
  // flops: H z (one FMA per stored H entry, kappa scaling per slot) and 9 FMAs per lambda of the pipelined CG;
  // per solve, one row of the local saddle inverse per interface slot, owned flux slot and pressure unknown; per
  // operator evaluation the local M and D blocks (D and D^T)
  double per_solve = 0.0;
  for (int cc = 0; cc < L.n_cells; ++cc) {
    const int nl = L.nloc(cc), mc = L.m[cc], n = nl + mc;
    int own = 0;
    for (int k = L.loc_off[cc]; k < L.loc_off[cc + 1]; ++k) own += own0[k];
    per_solve += 2.0 * n * ((if_off[cc + 1] - if_off[cc]) + own + mc);
  }
  c->sh->hyb_flops_per_iter[l] = 2.0 * (double)Hc.size() + 2.0 * D.nif + 18.0 * nlam;
  c->sh->hyb_flops_per_solve[l] = per_solve;
  c->sh->coarse_res_flops[l] = 2.0 * (double)L.Mloc.size() + 4.0 * (double)L.Dloc.size();
  // a trial: per flux unknown its b and slot ids, per owner slot its cell and the six parts read (ms, ds, pb of x and
  // of dx), per pressure unknown b and two parts; about 20 flops per owner slot (three FMAs and 1/kappa), 4 per
  // pressure unknown, 2 per unknown for the norm
  c->sh->coarse_trial_bytes[l] = 16.0 * D.nflux + (double)D.nyl * (4.0 + 48.0) + 24.0 * D.np;
  c->sh->coarse_trial_flops[l] = 20.0 * (double)D.nyl + 6.0 * D.np + 2.0 * D.nflux;
}

// Work buffers of coarse level l (per context).
void alloc_level(nlmg_ctx* c, int l) {
  const LevelDev& D = c->LD[l];
  const int nlam = D.nlam;
  CoarseBuf& B = c->CB[l];
  int nx = D.nflux + D.np;
  B.x = c->dalloc<double>(nx);
  B.b = c->dalloc<double>(nx);
  B.r = c->dalloc<double>(nx);
  B.dx = c->dalloc<double>(nx);
  B.nb = c->dalloc<double>(nx);
  B.xt2 = c->dalloc<double>(nx);
  B.xc = c->dalloc<double>(nx);
  B.yl = c->dalloc<double>(D.nyl);
  B.kapc = c->dalloc<double>(D.nc);
  B.ptmp = c->dalloc<double>(nx);
  B.ylam = c->dalloc<double>(D.nif);
  B.ydiag = c->dalloc<double>(D.nif);
  B.lam = c->dalloc<double>(nlam);
  B.lr = c->dalloc<double>(nlam);
  B.lz = c->dalloc<double>(nlam);
  B.lpa = c->dalloc<double>(nlam);
  B.lpb = c->dalloc<double>(nlam);
  B.lq = c->dalloc<double>(nlam);
  B.ldinv = c->dalloc<double>(nlam);
  B.xi = c->dalloc<double>(nlam);
  for (double** pp : {&B.hw, &B.hz, &B.hs, &B.hma, &B.hmb}) *pp = c->dalloc<double>(nlam);
  B.hsv = c->dalloc<double>((size_t)D.hs_n);
  for (LinParts* lp : {&B.base, &B.dir}) {
    lp->ms = c->dalloc<double>(D.nyl);
    lp->ds = c->dalloc<double>(D.nyl);
    lp->dr = c->dalloc<double>(D.np);
    lp->pb = c->dalloc<double>(D.nc);
  }
}

void upload_transfer(nlmg_ctx* c, int l) {
  const Level& L = c->H().levels[l];
  const Level& C = c->H().levels[l + 1];
  const Transfer& T = c->H().transfers[l];
  TransferDev& D = c->TD[l];
  D.na = C.n_cells;
  D.nrows = L.n_p();
  std::vector<int> roff(D.na + 1, 0), rows, pd_agg(D.nrows), pd_row(D.nrows);
  for (int a = 0; a < D.na; ++a) {
    int t = 0;
    for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
      int cc = T.agg_cells[k];
      for (int r = 0; r < L.m[cc]; ++r, ++t) {
        int i = L.p_off[cc] + r;
        rows.push_back(i);
        pd_agg[i] = a;
        pd_row[i] = t;
      }
    }
    roff[a + 1] = (int)rows.size();
  }
  D.rows_off = c->upload(roff);
  D.rows = c->upload(rows);
  D.pblk_off = c->upload(T.pblk_off);
  D.Pblk = c->upload(T.Pblk);
  D.mc = c->upload(C.m);
  D.pc_off = c->upload(C.p_off);
  D.pd_agg = c->upload(pd_agg);
  D.pd_row = c->upload(pd_row);
  D.ps_n = T.Ps.nrows;
  D.ps_off = c->upload(T.Ps.off);
  D.ps_col = c->upload(T.Ps.col);
  D.ps_val = c->upload(T.Ps.val);
  D.pst_n = T.PsT.nrows;
  D.pst_off = c->upload(T.PsT.off);
  D.pst_col = c->upload(T.PsT.col);
  D.pst_val = c->upload(T.PsT.val);
  D.qs_n = T.Qs.nrows;
  D.qs_off = c->upload(T.Qs.off);
  D.qs_col = c->upload(T.Qs.col);
  D.qs_val = c->upload(T.Qs.val);
}

// The multigrid preconditioner's structure on the first `levels` levels (read-only, shared by instances), with the
// algorithmic bytes of its phases: the per-step setup (fine values read and written, assembly contributions and the
// coarse blocks written), one V-cycle (level 0: each Chebyshev step and the residual read the SELL values and indices,
// b, x and write x, d; transfers read P; coarse levels the same with their blocks) and the Krylov vectors of one
// iteration.
void upload_mg(nlmg_ctx* c, int levels) {
  MgHost mh;
  std::string err;
  if (!mg_build_host(c->fm(), c->H(), levels, mh, err)) throw Error(NLMG_EUNSUPPORTED, err);
  MgDev& M = c->sh->MG;
  M.L = mh.L;
  M.N = mh.N;
  for (int l = 0; l < mh.L; ++l) {
    M.nc[l] = mh.nc[l];
    M.mb[l] = mh.mb[l];
    M.nblk[l] = mh.nblk[l];
    if (l >= 1) {
      M.rowptr[l] = c->upload(mh.rowptr[l]);
      M.col[l] = c->upload(mh.col[l]);
      M.dpos[l] = c->upload(mh.dpos[l]);
      M.mcnt[l] = c->upload(mh.mcnt[l]);
      M.asm_off[l] = c->upload(mh.asm_off[l]);
      M.asm_list[l] = c->upload(mh.asm_list[l]);
    }
    if (l + 1 < mh.L) {
      M.P[l] = c->upload(mh.P[l]);
      std::vector<__nv_bfloat16> pb(mh.P[l].size());
      for (size_t i = 0; i < pb.size(); ++i) pb[i] = __float2bfloat16(mh.P[l][i]);
      M.Pb[l] = c->upload(pb);
      M.agg[l] = c->upload(mh.agg[l]);
      M.ch_off[l] = c->upload(mh.ch_off[l]);
      M.ch[l] = c->upload(mh.ch[l]);
    }
  }
  const double N = mh.N, nnz = (double)c->sh->nnz_real;
  double setup = nnz * (8.0 + 4.0 + 4.0) + N * (8.0 + 12.0);   // Tval, indices read, FP32 values written; diagonals
  double vc = 0.0;
  const double fine_step = nnz * 8.0 + N * 20.0;                // SELL values + indices, b, x read, x, d written
  vc += (2.0 * kMgDegFine) * fine_step + N * 4.0 * mh.mb[1] * 2.0;   // steps, residual; P read twice
  for (int l = 1; l < mh.L; ++l) {
    const double mm = (double)mh.mb[l] * mh.mb[l];
    setup += (double)mh.asm_list[l].size() * 16.0 + mh.nblk[l] * mm * 4.0 * 2.0 + mh.nc[l] * mm * 4.0;
    if (l + 1 < mh.L) {
      const double cstep = mh.nblk[l] * (mm * 4.0 + 4.0) + mh.nc[l] * mm * 4.0 + mh.nc[l] * mh.mb[l] * 20.0;
      vc += (2.0 * kMgDegCoarse) * cstep + mh.P[l].size() * 4.0 * 2.0;
    } else {
      vc += (double)mh.nc[l] * mh.mb[l] * mh.nc[l] * mh.mb[l] * 4.0;
    }
  }
  c->sh->mg_bytes_setup = setup;
  c->sh->mg_bytes_vcycle = vc;
  c->sh->mg_bytes_iter = nnz * 12.0 + N * (8.0 * 10.0);   // A z (values, indices, z) and the FP64 vector updates
}

// ---------------------------------------------------------------------------------------------------------------
// level 0

double fine_eval(nlmg_ctx* c, const double* p, const double* dp, double s, FineState& out) {
  launch_kappa(c->st, c->F.N, p, dp, s, out.p, out.kap, nullptr, c->kind, c->a);
  int pi = c->prof_begin(2);
  launch_residual(c->st, c->F, out.p, out.kap, nullptr, c->g, c->rhs, out.R, nullptr, nullptr, nullptr, nullptr,
                  c->red(S_NORM2));
  c->prof_end(pi);
  c->fine_evals++;
  out.rn = std::sqrt(c->read_sc(S_NORM2));
  return out.rn;
}

// Algorithm 1 on level 0 from c->cur along dp (scaled by s0); the accepted trial becomes c->cur.
// Algorithm 1 on level 0. A trial whose residual norm is not finite counts as +infinity; if the trial the algorithm
// returns is not finite, the iterate is kept.
void backtrack0(nlmg_ctx* c, const double* dp, double s0) {
  const nlmg_options& o = c->opt;
  auto fin = [](double v) { return std::isfinite(v) ? v : HUGE_VAL; };
  double s = 1.0;
  int n = 0;
  double r_s = fin(fine_eval(c, c->cur.p, dp, s * s0, c->t1));
  while (r_s > c->cur.rn && n < o.bt_nmax) {
    double r_half = fin(fine_eval(c, c->cur.p, dp, 0.5 * s * s0, c->t2));
    if (r_half > o.bt_theta * r_s) break;
    s *= 0.5;
    ++n;
    r_s = r_half;
    std::swap(c->t1, c->t2);
  }
  if (r_s == HUGE_VAL) return;
  std::swap(c->cur, c->t1);
}

// Persistent CG on the frozen fine matrix (Tval, diagT): A dx = -R with symmetric Jacobi scaling; dx -> c->cx.
// lin_precision 0 runs it in FP64, 1 in FP32 (vectors and matrix; per-thread partial sums in FP32, block and grid
// sums in FP64).
int mg_pcg(nlmg_ctx* c, const double* R, const double* kap);
int mg_bicgstab(nlmg_ctx* c, const double* R, const double* kap);

int fine_pcg(nlmg_ctx* c, const double* R, const double* kap) {
  if (c->opt.lin_precond == 1) return mg_pcg(c, R, kap);
  GridSync gs{c->d_bar, &c->d_res->err, c->sm_cap};
  CK(cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned), c->st));
  CK(cudaMemsetAsync(c->d_res, 0, sizeof(PcgResult), c->st));
  launch_sdiag(c->st, c->F.N, c->diagT, c->sdiag);
  const bool fp32 = c->opt.lin_precision == 1;
  // FP64 at loose tolerances: pipelined CG (one grid barrier per iteration), register-resident when every thread
  // holds at most 4 cells. FP32: the pipelined CG with residual replacement every kReplace iterations (without it
  // the FP32 recurrences drift: measured 10,768 instead of 3,466 fine iterations on the 64^3 workload), registers
  // for at most 8 cells per thread; else the two-barrier CG in memory. Tight FP64 tolerances: the two-barrier CG, whose
  // updated residual tracks the true one more closely.
  constexpr int kReplace = 50;
  const bool pipe = !fp32 && c->lin_tol_eff >= 1e-6;
  int kind = 0;   // 0 two-barrier, 1 pipelined in memory, 2 pipelined in registers, 4 FP32 pipelined with
                  // residual replacement
  int pi;
  if (fp32) {
    launch_scale_sell<float>(c->st, c->F, c->Tval, c->sdiag, c->Ts32);
    pi = c->prof_begin(0);
    cudaError_t e = launch_fine_cg_rr32(c->st, c->F, c->Ts32, c->sdiag, R, -1.0, c->cx, c->fpa, c->fpb, c->fy,
                                        c->fq, c->fr, c->fs, c->d_partial, gs, std::max(c->lin_tol_eff, 1e-6),
                                        c->opt.lin_maxit, kReplace, c->d_res);
    kind = 4;
    if (e == cudaErrorNotSupported) {
      kind = 0;
      CK(launch_fine_cg<float>(c->st, c->F, c->Ts32, c->sdiag, R, -1.0, c->cx, c->fy, c->fr, c->fpa, c->fpb, c->fq,
                               c->d_partial, gs, std::max(c->lin_tol_eff, 1e-6), c->opt.lin_maxit, c->d_res));
    } else {
      CK(e);
    }
  } else {
    launch_scale_sell<double>(c->st, c->F, c->Tval, c->sdiag, c->Ts64);
    pi = c->prof_begin(0);
    cudaError_t e = cudaErrorNotSupported;
    if (pipe)
      e = launch_fine_cg_reg<double>(c->st, c->F, c->Ts64, c->sdiag, R, -1.0, c->cx, c->dv1, c->dv2, c->d_partial,
                                     gs, c->lin_tol_eff, c->opt.lin_maxit, c->d_res);
    if (e == cudaSuccess) {
      kind = 2;
    } else if (e != cudaErrorNotSupported) {
      CK(e);
    } else if (pipe) {
      kind = 1;
      CK(launch_fine_cg_pipe<double>(c->st, c->F, c->Ts64, c->sdiag, R, -1.0, c->cx, c->cz, c->cr, c->cpa, c->cpb,
                                     c->cq, c->dv1, c->dv2, c->d_partial, gs, c->lin_tol_eff, c->opt.lin_maxit,
                                     c->d_res));
    } else {
      CK(launch_fine_cg<double>(c->st, c->F, c->Ts64, c->sdiag, R, -1.0, c->cx, c->cz, c->cr, c->cpa, c->cpb,
                                c->cq, c->d_partial, gs, c->lin_tol_eff, c->opt.lin_maxit, c->d_res));
    }
  }
  c->last_fine_kind = kind;
  c->prof_end(pi);
  count_launch(1);
  CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(PcgResult), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_res->err) throw Error(NLMG_ETIMEOUT, "grid barrier wait gave up in the fine CG kernel");
  if (!std::isfinite(c->h_res->rr)) throw Error(NLMG_EDIVERGED, "non-finite value in the level-0 linear solve");
  const int it = c->h_res->iters;
  if (pi >= 0) {
    // Algorithmic bytes: per iteration the scaled matrix entries and their indices, then for the two-barrier CG
    // r read, p and q read and written, p, q, y, r read and y, r written (11 vectors); for the pipelined CG in
    // memory w, z, s, p, y, r read and z, s, p, y, r, w written (12 vectors); for the register-resident forms only
    // the exchanged vector (w, or r) gathered and written (2 vectors). The pipelined forms take one extra product
    // at the start. Once: b and
    // S read, y and r written, then S and y read and dx written. Gathered neighbour values are counted once.
    // Flops: one product (2 per stored entry) plus 6 FMAs per cell (two-barrier) or 9 (pipelined) per iteration.
    const double N = c->F.N, nnz = (double)c->sh->nnz_real, v = fp32 ? 4.0 : 8.0;
    const double nvec = kind >= 2 ? 2.0 : kind == 1 ? 12.0 : 11.0;
    const double per_it_b = (4.0 + v) * nnz + nvec * v * N;
    const bool pipelined = kind == 1 || kind == 2 || kind == 4;
    const double per_it_f = pipelined ? 2.0 * nnz + 18.0 * N : 2.0 * nnz + 12.0 * N;   // an FMA counts 2
    c->prof.bytes[0] += (8.0 + 8.0) * N + 2.0 * v * N + 8.0 * N + v * N + 8.0 * N + (pipelined ? per_it_b : 0.0) +
                        it * per_it_b;
    c->prof.flops[0] += it * per_it_f;
  }
  c->lin_iters += it;
  c->lin_iters_level[0] += it;
  return it;
}

void alloc_newton(nlmg_ctx* c) {
  if (c->Joff) return;
  const int N = c->F.N;
  c->Joff = c->dalloc<double>(c->F.nnz);
  c->jdinv = c->dalloc<double>(N);
  c->gV = c->dalloc<double>((size_t)(nlmg_ctx::kGmresM + 1) * N);
  c->gw = c->dalloc<double>(N);
  c->gu = c->dalloc<double>(N);
  c->gr = c->dalloc<double>(N);
  c->gh = c->dalloc<double>(3 * 64);
  CK(cudaMallocHost(&c->h_gh, 3 * 64 * sizeof(double)));
  c->Js = c->dalloc<double>(c->F.nnz);
  c->jdS = c->dalloc<double>(N);
  c->jsS = c->dalloc<double>(N);
}

// The exact Jacobian at c->cur.p (Sec. 3.3.2 on level 0): kappa and kappa' per cell, the residual kernel's
// Jacobian diagonal and off-diagonal entries (SELL layout), the frozen diagonal d and the Jacobi weights
// 1 / max(J_KK, d_K / 2).
void newton_linearize(nlmg_ctx* c) {
  alloc_newton(c);
  const int N = c->F.N;
  launch_kappa(c->st, N, c->cur.p, nullptr, 0.0, c->cur.p, c->t2.kap, c->dkap, c->kind, c->a);
  launch_residual(c->st, c->F, c->cur.p, c->t2.kap, c->dkap, c->g, c->rhs, c->t2.R,
                  c->opt.lin_precond == 1 ? c->Tval : nullptr, nullptr, c->diagT, c->jdiag, c->red(S_NORM2B),
                  c->Joff);
  launch_jacobi_dinv(c->st, N, c->jdiag, c->diagT, c->jdinv);
}

// Persistent FP64 BiCGStab on the Jacobi-scaled Newton system J dx = -R (J from newton_linearize) to newton_tol_eff;
// dx -> c->cx.
int fine_bicgstab(nlmg_ctx* c, const double* R) {
  if (c->opt.lin_precond == 1) return mg_bicgstab(c, R, c->t2.kap);
  GridSync gs{c->d_bar, &c->d_res->err, c->sm_cap};
  CK(cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned), c->st));
  CK(cudaMemsetAsync(c->d_res, 0, sizeof(PcgResult), c->st));
  launch_scale_jac(c->st, c->F, c->jdiag, c->Joff, c->jdinv, c->Js, c->jdS, c->jsS);
  const int pi = c->prof_begin(3);
  CK(launch_fine_bicgstab(c->st, c->F, c->Js, c->jdS, c->jsS, R, -1.0, c->cx, c->gV, c->d_partial, gs,
                          c->newton_tol_eff, c->opt.lin_maxit, c->d_res));
  c->prof_end(pi);
  count_launch(1);
  CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(PcgResult), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_res->err) throw Error(NLMG_ETIMEOUT, "grid barrier wait gave up in the fine BiCGStab kernel");
  if (!std::isfinite(c->h_res->rr)) throw Error(NLMG_EDIVERGED, "non-finite value in the level-0 Newton solve");
  const int it = c->h_res->iters;
  if (pi >= 0) {
    // Algorithmic bytes: once, b and S read, y, r, rh, p written, then S and y read and dx written (10 vectors).
    // Per iteration the scaled Jacobian (values, indices, diagonal) twice, and the vectors of the five passes:
    // p gathered, rh read, v written; r, v read, s written; s gathered, t written; s, y, p, t, rh read, y, r
    // written; r, p, v read, p written (19 vectors). Flops: two products (2 per stored entry, diagonal included)
    // and 11 FMAs per cell per iteration.
    const double N = c->F.N, nnz = (double)c->sh->nnz_real;
    c->prof.bytes[3] += 10.0 * 8.0 * N + it * (2.0 * (12.0 * nnz + 8.0 * N) + 19.0 * 8.0 * N);
    c->prof.flops[3] += it * (4.0 * (nnz + N) + 22.0 * N);
  }
  c->lin_iters += it;
  c->lin_iters_level[0] += it;
  return it;
}

// Restarted GMRES(30) with right Jacobi preconditioning for J dx = -R (Sec. 3.3.2's linear system on level 0, the
// single-level Newton baseline); classical Gram-Schmidt with one reorthogonalisation. dx -> c->cx.
int fine_gmres(nlmg_ctx* c, const double* R) {
  const int N = c->F.N, m = nlmg_ctx::kGmresM;
  double* V = c->gV;
  double* hA = c->gh;            // first Gram-Schmidt coefficients
  double* hB = c->gh + 64;       // reorthogonalisation coefficients
  auto norm = [&](double* x) {   // ||x|| (orthogonalisation against no vectors)
    launch_orth_update(c->st, N, 0, V, hA, x, c->red(S_NORM2B));
    return std::sqrt(c->read_sc(S_NORM2B));
  };
  CK(cudaMemsetAsync(c->gu, 0, (size_t)N * sizeof(double), c->st));
  launch_scale_vec(c->st, N, R, -1.0, c->gr);       // r = b = -R (u = 0)
  const double beta0 = norm(c->gr);
  double beta = beta0;
  int total = 0;
  if (!(beta0 > 0.0)) {
    CK(cudaMemsetAsync(c->cx, 0, (size_t)N * sizeof(double), c->st));
    return 0;
  }
  const double tol = c->lin_tol_eff * beta0;
  {
    const double one = 1.0;
    CK(cudaMemcpyAsync(c->gh + 191, &one, sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gvec(m + 1);
  while (true) {
    launch_scale_vec(c->st, N, c->gr, 1.0 / beta, V);
    std::fill(gvec.begin(), gvec.end(), 0.0);
    gvec[0] = beta;
    int j = 0;
    double res = beta;
    for (; j < m; ++j) {
      double* vj1 = V + (size_t)(j + 1) * N;
      launch_jac_apply(c->st, c->F, c->jdiag, c->Joff, c->jdinv, V + (size_t)j * N, c->gw);
      launch_mdot(c->st, N, j + 1, V, c->gw, c->d_partial, c->d_cnt + 8, hA);
      launch_orth_update(c->st, N, j + 1, V, hA, c->gw, c->red(S_NORM2B));
      launch_mdot(c->st, N, j + 1, V, c->gw, c->d_partial, c->d_cnt + 8, hB);
      launch_orth_update(c->st, N, j + 1, V, hB, c->gw, c->red(S_NORM2B));
      CK(cudaMemcpyAsync(c->h_gh, c->gh, 128 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      const double wn = std::sqrt(c->read_sc(S_NORM2B));   // synchronizes the stream
      for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = c->h_gh[k] + c->h_gh[64 + k];
      H[(size_t)(j + 1) * m + j] = wn;
      for (int k = 0; k < j; ++k) {   // previous rotations
        const double a = H[(size_t)k * m + j], b = H[(size_t)(k + 1) * m + j];
        H[(size_t)k * m + j] = cs[k] * a + sn[k] * b;
        H[(size_t)(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
      }
      const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      const double r = std::hypot(a, b);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b / r : 0.0;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gvec[j + 1] = -sn[j] * gvec[j];
      gvec[j] = cs[j] * gvec[j];
      res = std::fabs(gvec[j + 1]);
      ++total;
      if (wn > 0.0) launch_scale_vec(c->st, N, c->gw, 1.0 / wn, vj1);
      if (res <= tol || wn == 0.0 || total >= c->opt.lin_maxit) {
        ++j;
        break;
      }
    }
    // y = H(0:j, 0:j)^-1 g ; u += V y
    std::vector<double> y(j, 0.0);
    for (int k = j - 1; k >= 0; --k) {
      double v = gvec[k];
      for (int q = k + 1; q < j; ++q) v -= H[(size_t)k * m + q] * y[q];
      y[k] = H[(size_t)k * m + k] != 0.0 ? v / H[(size_t)k * m + k] : 0.0;
    }
    CK(cudaMemcpyAsync(c->gh + 128, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    launch_gmres_combine(c->st, N, j, V, c->gh + 128, nullptr, c->gw);   // u += V y
    launch_axpy(c->st, N, c->gu, 1.0, c->gw, c->gu);
    if (res <= tol || total >= c->opt.lin_maxit) break;
    // true residual r = b - J D u
    launch_jac_apply(c->st, c->F, c->jdiag, c->Joff, c->jdinv, c->gu, c->gw);
    launch_scale_vec(c->st, N, c->gw, -1.0, c->gr);       // r = -J D u ...
    launch_axpy(c->st, N, c->gr, -1.0, R, c->gr);         // ... - R = b - J D u
    beta = norm(c->gr);
    if (!(beta > tol)) break;
  }
  // dx = D u
  launch_gmres_combine(c->st, N, 1, c->gu, c->gh + 191, c->jdinv, c->cx);   // dx = D u (weight gh[191] = 1)
  c->lin_iters += total;
  c->lin_iters_level[0] += total;
  return total;
}

// One single-level Newton step (Sec. 3.3.2 on level 0): exact Jacobian, GMRES, clamp, Algorithm 1.
void newton_step(nlmg_ctx* c) {
  const int N = c->F.N;
  newton_linearize(c);
  fine_gmres(c, c->cur.R);
  double s0 = 1.0;
  if (c->opt.dp_clamp > 0) {
    launch_max_abs(c->st, N, c->cx, c->red(S_MAX));
    double mx = c->read_sc(S_MAX);
    if (mx > c->opt.dp_clamp) s0 = c->opt.dp_clamp / mx;
  }
  backtrack0(c, c->cx, s0);
}

// A Newton smoothing step that leaves more than this fraction of the residual it started from shows that the
// iterate is outside Newton's region of fast convergence: the rest of the solve takes Picard steps.
constexpr double kNewtonKeep = 0.5;

// One smoothing step on level 0 (Picard, Newton or nonlinear Jacobi), then the clamp and Algorithm 1. With the
// Picard-then-Newton smoother the step is a Newton step once ||R(p_k)|| <= newton_switch ||R(p_0)||, unless an
// earlier Newton step of the solve failed to halve the residual.
void smooth0(nlmg_ctx* c, int nu) {
  const nlmg_options& o = c->opt;
  const int N = c->F.N;
  const double* dp = nullptr;
  const double rn_in = c->cur.rn;
  const bool newton =
      o.smoother == NLMG_SMOOTH_PICARD_NEWTON && !c->newton_off && rn_in <= o.newton_switch * c->r0_ref;
  if (newton) {
    newton_linearize(c);
    fine_bicgstab(c, c->cur.R);
    dp = c->cx;
    c->newton_steps++;
  } else if (o.smoother == NLMG_SMOOTH_PICARD || o.smoother == NLMG_SMOOTH_PICARD_NEWTON) {
    launch_residual(c->st, c->F, c->cur.p, c->cur.kap, nullptr, c->g, c->rhs, c->t2.R, c->Tval, c->dinv, c->diagT,
                    nullptr, c->red(S_NORM2B));
    fine_pcg(c, c->cur.R, c->cur.kap);
    dp = c->cx;
  } else {
    // nu sweeps q <- q - omega R(q) / max(J_qq, d_q / 2) from q = p, then dp = q - p
    double* q = c->cpa;
    double* qn = c->cpb;
    CK(cudaMemcpyAsync(q, c->cur.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    for (int k = 0; k < nu; ++k) {
      launch_kappa(c->st, N, q, nullptr, 0.0, q, c->t2.kap, c->dkap, c->kind, c->a);
      launch_residual(c->st, c->F, q, c->t2.kap, c->dkap, c->g, c->rhs, c->t2.R, nullptr, nullptr, c->diagT,
                      c->jdiag, c->red(S_NORM2B));
      launch_jacobi_update(c->st, N, q, c->t2.R, c->jdiag, c->diagT, o.omega, qn);
      std::swap(q, qn);
      c->fine_evals++;
    }
    launch_sub(c->st, N, q, c->cur.p, c->cx);
    dp = c->cx;
  }
  double s0 = 1.0;
  if (o.dp_clamp > 0) {
    launch_max_abs(c->st, N, dp, c->red(S_MAX));
    double mx = c->read_sc(S_MAX);
    if (mx > o.dp_clamp) s0 = o.dp_clamp / mx;
  }
  backtrack0(c, dp, s0);
  if (newton && !(c->cur.rn <= kNewtonKeep * rn_in)) c->newton_off = true;
}

// ---------------------------------------------------------------------------------------------------------------
// coarse levels

// r = A^l(x) - b (b may be null), kapc; returns ||r||.
double coarse_res(nlmg_ctx* c, int l, const double* x, const double* b, double* r) {
  const LevelDev& L = c->LD[l];
  CoarseBuf& B = c->CB[l];
  launch_coarse_cell(c->st, L, x, x + L.nflux, b ? b + L.nflux : nullptr, B.yl, r + L.nflux, B.kapc, c->kind, c->a,
                     c->red(S_NORM2));
  launch_coarse_flux(c->st, L, B.yl, b, r, c->red(S_NORM2B));
  double v0, v1;
  c->read_sc2(S_NORM2, v0, v1);
  return std::sqrt(v0 + v1);
}

// x_{l+1} = Q x_l, b_{l+1} = A_{l+1}(x_{l+1}) - P^T r_l (r_l = [r_sigma; r_p] of level l >= 1 in CB[l].r)
void make_coarse_problem(nlmg_ctx* c, int l) {
  const TransferDev& T = c->TD[l];
  const LevelDev& C = c->LD[l + 1];
  CoarseBuf& Bc = c->CB[l + 1];
  if (l == 0) {
    launch_kappa(c->st, c->F.N, c->cur.p, nullptr, 0.0, c->cur.p, c->cur.kap, nullptr, c->kind, c->a);
    launch_fine_flux(c->st, c->F, c->cur.p, c->cur.kap, c->g, c->sig0);
    launch_csr(c->st, T.qs_n, T.qs_off, T.qs_col, T.qs_val, c->sig0, Bc.x, 1.0, 0.0);
    // projection of p and restriction of the mixed pressure residual -R
    launch_restrict_p(c->st, T, c->cur.p, Bc.x + C.nflux, 1.0, c->cur.R, Bc.ptmp + C.nflux);
    coarse_res(c, l + 1, Bc.x, nullptr, Bc.b);
    // b_p += P^T R   (R r^0 = [0; P^T (-R)])
    launch_axpy(c->st, C.np, Bc.b + C.nflux, 1.0, Bc.ptmp + C.nflux, Bc.b + C.nflux);
  } else {
    const LevelDev& L = c->LD[l];
    CoarseBuf& B = c->CB[l];
    launch_csr(c->st, T.qs_n, T.qs_off, T.qs_col, T.qs_val, B.x, Bc.x, 1.0, 0.0);
    launch_restrict_p(c->st, T, B.x + L.nflux, Bc.x + C.nflux, 1.0, B.r + L.nflux, Bc.ptmp + C.nflux);
    coarse_res(c, l + 1, Bc.x, nullptr, Bc.b);
    launch_csr(c->st, T.pst_n, T.pst_off, T.pst_col, T.pst_val, B.r, Bc.b, -1.0, 1.0);
    launch_axpy(c->st, C.np, Bc.b + C.nflux, -1.0, Bc.ptmp + C.nflux, Bc.b + C.nflux);
  }
  CK(cudaMemcpyAsync(Bc.xc, Bc.x, (size_t)(C.nflux + C.np) * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
}

// One launch of the fused coarse Picard step on level l (see launch_coarse_step): optional Algorithm 1 along B.dx
// from s = 1, then up to nsteps Picard steps, then optionally the residual at the final x. B.rn is updated.
// One launch of the fused coarse step on level l: [Algorithm 1 along B.dx,] nsteps Picard steps; leaves x, r = A(x) - b,
// -r and kappa per cell at the final x, and ||r|| in B.rn.
void coarse_step(nlmg_ctx* c, int l, bool backtrack_first, int nsteps, bool coarsest) {
  const LevelDev& L = c->LD[l];
  CoarseBuf& B = c->CB[l];
  CoarseStepParams P{};
  P.kind = c->kind;
  P.a = c->a;
  P.dp_clamp = c->opt.dp_clamp;
  P.bt_nmax = c->opt.bt_nmax;
  P.bt_theta = c->opt.bt_theta;
  P.backtrack_first = backtrack_first ? 1 : 0;
  P.rn_in = B.rn;
  P.nsteps = nsteps;
  P.coarsest = coarsest ? 1 : 0;
  P.tol_rel = c->opt.coarsest_tol > 0.0 ? c->opt.coarsest_tol : c->tol_rel;
  P.tol_abs = c->tol_abs;
  P.maxit = c->opt.lin_maxit;
  GridSync gs{c->d_bar, &c->d_res->err, c->sm_cap};
  CK(cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned), c->st));
  CK(cudaMemsetAsync(c->d_res, 0, sizeof(PcgResult), c->st));
  CoarseStepResult* dres = (CoarseStepResult*)(c->d_res + 1);
  CK(cudaMemsetAsync(dres, 0, sizeof(CoarseStepResult), c->st));
  const int kid = coarsest ? 4 : 1;   // profile id: the coarsest solve apart from the other coarse steps
  int pi = c->prof_begin(kid);
  // FP64 whatever lin_precision is: the coarse levels are latency bound, FP32 would save nothing there. Pipelined
  // hybridized CG at loose tolerances; the two-synchronisation CG when a tight solve is asked for.
  P.lin_tol = coarsest ? c->coarsest_lin_tol_eff : c->coarse_lin_tol_eff;
  const bool pipe = P.lin_tol >= 1e-6;
  CoarseStepBufs<double> Bd{B.x, B.b, B.r, B.nb, B.dx, B.kapc, B.base, B.dir, B.ylam, B.ydiag,
                            B.lam, B.lr, B.lz, B.lpa, B.lpb, B.lq, B.ldinv,
                            pipe ? HybPipeBufs<double>{B.hw, B.hz, B.hs, B.hma, B.hmb} : HybPipeBufs<double>{},
                            B.hsv};
  bool sell = false;
  CK(launch_coarse_step<double>(c->st, L, L.Hc, L.Sinv, Bd, P, c->d_partial, gs, dres, &sell));
  c->prof_end(pi);
  count_launch(1);
  CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(PcgResult) + sizeof(CoarseStepResult), cudaMemcpyDeviceToHost,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->h_res->err) throw Error(NLMG_ETIMEOUT, "grid barrier wait gave up in the coarse step kernel");
  const CoarseStepResult& R = *(const CoarseStepResult*)(c->h_res + 1);
  if (R.bad)
    throw Error(NLMG_EDIVERGED, std::string("non-finite value in the ") +
                                    (R.bad == 1 ? "residual" : "hybridized linear solve") + " of coarse level " +
                                    std::to_string(l));
  B.rn = R.rn;
  if (pi >= 0) {
    const double per_iter = sell ? c->sh->hyb_bytes_per_iter_sell[l] : c->sh->hyb_bytes_per_iter[l];
    c->prof.bytes[kid] += (double)R.iters * per_iter +
                          (double)R.res_evals * c->sh->coarse_res_bytes[l] +
                          (double)(R.trials + R.steps + 1) * c->sh->coarse_trial_bytes[l];
    c->prof.flops[kid] += (double)R.iters * c->sh->hyb_flops_per_iter[l] +
                          (double)R.steps * c->sh->hyb_flops_per_solve[l] +
                          (double)R.res_evals * c->sh->coarse_res_flops[l] +
                          (double)(R.trials + R.steps + 1) * c->sh->coarse_trial_flops[l];
  }
  c->lin_iters += R.iters;
  c->lin_iters_level[l] += R.iters;
}

void coarse_cycle(nlmg_ctx* c, int l) {
  const nlmg_options& o = c->opt;
  CoarseBuf& B = c->CB[l];
  const LevelDev& L = c->LD[l];
  if (l == c->nlev() - 1) {
    coarse_step(c, l, false, o.coarsest_steps, true);
    return;
  }
  coarse_step(c, l, false, 1, false);   // pre-smoothing; leaves r at the smoothed x for the restriction
  make_coarse_problem(c, l);
  coarse_cycle(c, l + 1);
  const LevelDev& C = c->LD[l + 1];
  CoarseBuf& Bc = c->CB[l + 1];
  const TransferDev& T = c->TD[l];
  launch_sub(c->st, C.nflux + C.np, Bc.x, Bc.xc, Bc.ptmp);
  launch_csr(c->st, T.ps_n, T.ps_off, T.ps_col, T.ps_val, Bc.ptmp, B.dx, 1.0, 0.0);
  launch_prolong_p(c->st, T, Bc.ptmp + C.nflux, B.dx + L.nflux);
  coarse_step(c, l, true, 1, false);   // Algorithm 1 along the correction, then post-smoothing
}

// One FAS cycle from level 0 (Algorithm 2). Returns true if it stopped after pre-smoothing.
bool vcycle(nlmg_ctx* c, double r0, double tol_rel, double tol_abs) {
  const nlmg_options& o = c->opt;
  smooth0(c, o.nu_pre);
  if (c->cur.rn <= tol_rel * r0 || c->cur.rn <= tol_abs) return true;
  if (c->nlev() > 1) {
    make_coarse_problem(c, 0);
    coarse_cycle(c, 1);
    const LevelDev& C = c->LD[1];
    CoarseBuf& Bc = c->CB[1];
    launch_sub(c->st, C.nflux + C.np, Bc.x, Bc.xc, Bc.ptmp);
    launch_prolong_p(c->st, c->TD[0], Bc.ptmp + C.nflux, c->fdp);
    backtrack0(c, c->fdp, 1.0);
  }
  smooth0(c, o.nu_post);
  return false;
}

// Nonlinear cascadic start (Sec. 4.2): the FAS coarse problems of Algorithm 2 formed top-down at the current
// level-0 iterate with no smoothing, then solved from the coarsest level up, each by up to coarsest_steps Picard
// steps that stop like the coarsest solve, from the point its finer level projected; each level's correction
// y - Qx is carried to the finer level with Algorithm 1, the level-0 one too. Leaves cur (p, R, ||R||).
void cascade(nlmg_ctx* c) {
  const int nl = c->nlev();
  if (nl < 2) return;
  const nlmg_options& o = c->opt;
  make_coarse_problem(c, 0);
  for (int l = 1; l + 1 < nl; ++l) {
    CoarseBuf& B = c->CB[l];
    B.rn = coarse_res(c, l, B.x, B.b, B.r);   // r = A(x) - b at the projected x, restricted below
    make_coarse_problem(c, l);
  }
  coarse_step(c, nl - 1, false, o.coarsest_steps, true);
  for (int l = nl - 2; l >= 1; --l) {
    const LevelDev& L = c->LD[l];
    const LevelDev& C = c->LD[l + 1];
    CoarseBuf& B = c->CB[l];
    CoarseBuf& Bc = c->CB[l + 1];
    const TransferDev& T = c->TD[l];
    launch_sub(c->st, C.nflux + C.np, Bc.x, Bc.xc, Bc.ptmp);
    launch_csr(c->st, T.ps_n, T.ps_off, T.ps_col, T.ps_val, Bc.ptmp, B.dx, 1.0, 0.0);
    launch_prolong_p(c->st, T, Bc.ptmp + C.nflux, B.dx + L.nflux);
    coarse_step(c, l, true, o.coarsest_steps, true);   // Algorithm 1 along the correction, then the level solve
  }
  const LevelDev& C = c->LD[1];
  CoarseBuf& Bc = c->CB[1];
  launch_sub(c->st, C.nflux + C.np, Bc.x, Bc.xc, Bc.ptmp);
  launch_prolong_p(c->st, c->TD[0], Bc.ptmp + C.nflux, c->fdp);
  backtrack0(c, c->fdp, 1.0);
}

void alloc_fine(nlmg_ctx* c) {
  const int N = c->F.N;
  c->f = c->dalloc<double>(N);
  c->g = c->dalloc<double>(c->fm().n_faces);
  c->rhs = c->dalloc<double>(N);
  c->dkap = c->dalloc<double>(N);
  c->Tval = c->dalloc<double>(c->F.nnz);
  c->dinv = c->dalloc<double>(N);
  c->diagT = c->dalloc<double>(N);
  c->jdiag = c->dalloc<double>(N);
  c->sig0 = c->dalloc<double>(c->F.nflux);
  c->fdp = c->dalloc<double>(N);
  c->cx = c->dalloc<double>(N);
  c->cr = c->dalloc<double>(N);
  c->cz = c->dalloc<double>(N);
  c->cpa = c->dalloc<double>(N);
  c->cpb = c->dalloc<double>(N);
  c->cq = c->dalloc<double>(N);
  c->sdiag = c->dalloc<double>(N);
  c->dv1 = c->dalloc<double>(N);
  c->dv2 = c->dalloc<double>(N);
  c->Ts64 = c->dalloc<double>(c->F.nnz);
  c->Ts32 = c->dalloc<float>(c->F.nnz);
  for (float** pp : {&c->fy, &c->fr, &c->fpa, &c->fpb, &c->fq, &c->fs}) *pp = c->dalloc<float>(N);
  for (FineState* s : {&c->cur, &c->t1, &c->t2}) {
    s->p = c->dalloc<double>(N);
    s->kap = c->dalloc<double>(N);
    s->R = c->dalloc<double>(N);
  }
}

// Work buffers of the multigrid preconditioner (when the shared part holds one).
void alloc_mg(nlmg_ctx* c) {
  const MgDev& M = c->sh->MG;
  if (M.L == 0) return;
  MgWork& W = c->mg;
  const int N = c->F.N;
  {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    W.grid0 = std::max(1, sms) * 8;   // the level-0 kernels use at most 32 registers: 8 blocks of 256 per SM
  }
  W.a0off = c->dalloc<float>(c->F.nnz);
  W.a0diag = c->dalloc<float>(N);
  W.a0dinv = c->dalloc<float>(N);
  for (int l = 0; l < M.L; ++l) {
    const size_t n = l == 0 ? (size_t)N : (size_t)M.nc[l] * M.mb[l];
    W.x[l][0] = c->dalloc<float>(n);
    W.x[l][1] = c->dalloc<float>(n);
    W.b[l] = c->dalloc<float>(n);
    W.d[l] = c->dalloc<float>(n);
    if (l >= 1) {
      W.aval[l] = c->dalloc<float>((size_t)M.nblk[l] * M.mb[l] * M.mb[l]);
      W.dinv[l] = c->dalloc<float>((size_t)M.nc[l] * M.mb[l] * M.mb[l]);
    }
  }
  const int nco = M.nc[M.L - 1] * M.mb[M.L - 1];
  W.cinv = c->dalloc<float>((size_t)nco * nco);
  W.lam = c->dalloc<float>(kMgMaxLevels);
  W.coef = c->dalloc<float>(kMgMaxLevels * kMgMaxDeg * 2);
  W.kx = c->cx;
  W.z[0] = c->dalloc<float>(N);
  for (double** pp : {&W.kr, &W.kp, &W.kq, &W.kb, &W.kv, &W.ks, &W.kt, &W.krh, &W.kpp}) *pp = c->dalloc<double>(N);
  W.part = c->dalloc<double>((size_t)2 * 1024);
  W.sc = c->dalloc<MgScal>(1);
  CK(cudaMemsetAsync(W.sc, 0, sizeof(MgScal), c->st));
  CK(cudaMallocHost(&W.h_sc, sizeof(MgScal)));
  W.tail = c->dalloc<MgTailTab>(1);
  mg_fill_tail(c->st, M, W);
  CK(cudaGetLastError());
  mg_set_smem_limits();
}

// Transfers of the preconditioner in BF16 (lin_precision = 2) or FP32, and the level size from which the block levels
// run row-parallel (mg_row_cells); graphs captured with other choices are dropped and captured again.
void mg_select_precision(nlmg_ctx* c) {
  MgWork& W = c->mg;
  W.bf16 = c->opt.lin_precision == 2 ? 1 : 0;
  W.row_cells = c->opt.mg_row_cells;
  if ((W.graphs_bf16 != -1 && W.graphs_bf16 != W.bf16) || (W.graphs_row_cells != -1 && W.graphs_row_cells != W.row_cells)) {
    for (cudaGraphExec_t* g : {&W.g_pcg[0], &W.g_pcg[1], &W.g_bicg[0], &W.g_bicg[1], &W.g_apply})
      if (*g) {
        CK(cudaGraphExecDestroy(*g));
        *g = nullptr;
      }
  }
  W.graphs_bf16 = W.bf16;
  W.graphs_row_cells = W.row_cells;
}

// Reads the scalars of the last multigrid Krylov solve; throws on a non-finite value.
int mg_finish(nlmg_ctx* c, const char* what) {
  MgWork& W = c->mg;
  CK(cudaMemcpyAsync(W.h_sc, W.sc, sizeof(MgScal), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (W.h_sc->bad) throw Error(NLMG_EDIVERGED, std::string("non-finite value in the level-0 ") + what);
  return W.h_sc->it;
}

// Tolerance and iteration cap of the next multigrid Krylov solve (read by its graphs on the device).
void mg_set_limits(nlmg_ctx* c, double tol) {
  MgWork& W = c->mg;
  W.h_sc->tol2 = tol * tol;
  W.h_sc->maxit = c->opt.lin_maxit;
  CK(cudaMemcpyAsync(&W.sc->tol2, &W.h_sc->tol2, sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(&W.sc->maxit, &W.h_sc->maxit, sizeof(int), cudaMemcpyHostToDevice, c->st));
}

// Level-0 Picard system A(kappa(p)) dx = -R (A from the last residual launch with Tval / diagT; kappa per cell in
// kap for the Dirichlet terms of the Galerkin operators) by CG preconditioned with one multigrid V-cycle; dx -> c->cx.
// Stops at ||S r|| <= lin_tol ||S r_0|| (S = diag(A)^-1/2, the test of the Jacobi-preconditioned CG) or lin_maxit.
int mg_pcg(nlmg_ctx* c, const double* R, const double* kap) {
  const MgDev& M = c->sh->MG;
  MgWork& W = c->mg;
  mg_select_precision(c);
  const int ps = c->prof_begin(7);
  mg_enqueue_setup(c->st, M, c->F, W, c->Tval, c->diagT, kap);
  c->prof_end(ps);
  const int pi = c->prof_begin(5);
  CK(cudaMemcpyAsync(W.kb, R, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  mg_set_limits(c, c->lin_tol_eff);
  if (!W.g_pcg[0]) CK(mg_capture_pcg(c->st, M, c->F, W, c->Tval, c->diagT, W.g_pcg));
  CK(cudaGraphLaunch(W.g_pcg[0], c->st));
  CK(cudaGraphLaunch(W.g_pcg[1], c->st));
  c->prof_end(pi);
  const int it = mg_finish(c, "multigrid-preconditioned CG");
  const int V = mg_vcycle_kernels(M);
  count_launch(1 + std::max(it, 1) * (2 + V));   // the start, then one loop body per iteration
  if (pi >= 0) {
    c->prof.bytes[5] += (double)it * (c->sh->mg_bytes_vcycle + c->sh->mg_bytes_iter);
    c->prof.bytes[7] += c->sh->mg_bytes_setup;
  }
  c->lin_iters += it;
  c->lin_iters_level[0] += it;
  return it;
}

// Level-0 Newton system J dx = -R (J from newton_linearize, preconditioner from the Picard matrix at the same point)
// by right-preconditioned BiCGStab with one V-cycle per preconditioning; stops at ||W r|| <= newton_lin_tol ||W r_0||
// with W^2 = 1 / max(J_KK, d_K / 2), the test of the Jacobi-scaled BiCGStab; dx -> c->cx.
int mg_bicgstab(nlmg_ctx* c, const double* R, const double* kap) {
  const MgDev& M = c->sh->MG;
  MgWork& W = c->mg;
  mg_select_precision(c);
  const int ps = c->prof_begin(7);
  mg_enqueue_setup(c->st, M, c->F, W, c->Tval, c->diagT, kap);
  c->prof_end(ps);
  const int pi = c->prof_begin(6);
  CK(cudaMemcpyAsync(W.kb, R, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  mg_set_limits(c, c->newton_tol_eff);
  if (!W.g_bicg[0]) CK(mg_capture_bicgstab(c->st, M, c->F, W, c->jdiag, c->Joff, c->jdinv, W.g_bicg));
  CK(cudaGraphLaunch(W.g_bicg[0], c->st));
  CK(cudaGraphLaunch(W.g_bicg[1], c->st));
  c->prof_end(pi);
  const int it = mg_finish(c, "multigrid-preconditioned BiCGStab");
  const int V = mg_vcycle_kernels(M);
  count_launch(1 + std::max(it, 1) * (5 + 2 * V));
  if (pi >= 0) {
    c->prof.bytes[6] += (double)(2 * it) * c->sh->mg_bytes_vcycle + (double)it * 2.0 * c->sh->mg_bytes_iter;
    c->prof.bytes[7] += c->sh->mg_bytes_setup;
  }
  c->lin_iters += it;
  c->lin_iters_level[0] += it;
  return it;
}

nlmg_status fail(nlmg_ctx* c, nlmg_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

template <class F>
nlmg_status guarded(nlmg_ctx* c, F&& fn) {
  if (!c) return NLMG_EINVAL;
  try {
    return fn();
  } catch (const Error& e) {
    return fail(c, e.code, e.what());
  } catch (const std::exception& e) {
    return fail(c, NLMG_EINVAL, e.what());
  }
}

void set_data_dev(nlmg_ctx* c, const double* f_dev, const double* g_dev) {
  if (f_dev != c->f)
    CK(cudaMemcpyAsync(c->f, f_dev, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (g_dev != c->g)
    CK(cudaMemcpyAsync(c->g, g_dev, (size_t)c->fm().n_faces * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  launch_rhs(c->st, c->F, c->f, c->g, c->rhs);
  c->have_data = true;
}

void set_data_host(nlmg_ctx* c, const double* f, const double* g) {
  CK(cudaMemcpyAsync(c->f, f, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->g, g, (size_t)c->fm().n_faces * sizeof(double), cudaMemcpyHostToDevice, c->st));
  set_data_dev(c, c->f, c->g);
}

// Full solve on device data already set; x0 device pointer or null. Returns status.
// mode: 0 FAS cycles, 1 single-level Picard steps, 2 single-level Newton steps
nlmg_status solve_core(nlmg_ctx* c, const double* x0_dev, double tol_rel, double tol_abs, int max_cycles,
                       double* p_dev, nlmg_report* rep, int mode) {
  const bool picard_only = mode == 1;
  const int N = c->F.N;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, c->st));
  c->fine_evals = 0;
  c->lin_iters = 0;
  c->newton_steps = 0;
  for (auto& v : c->lin_iters_level) v = 0;
  const long long launches0 = launch_count_thread();
  c->tol_rel = tol_rel;
  c->tol_abs = tol_abs;
  c->reset_inner_tols();
  if (x0_dev)
    CK(cudaMemcpyAsync(c->cur.p, x0_dev, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  else
    CK(cudaMemsetAsync(c->cur.p, 0, (size_t)N * sizeof(double), c->st));
  double r0 = fine_eval(c, c->cur.p, nullptr, 0.0, c->cur);
  c->r0_ref = r0;
  c->newton_off = false;
  nlmg_report R{};
  R.res0 = r0;
  R.history[0] = r0;
  R.history_len = 1;
  int cycles = 0;
  bool early = false;
  nlmg_status st = NLMG_OK;
  const int saved_smoother = c->opt.smoother;
  if (picard_only) c->opt.smoother = NLMG_SMOOTH_PICARD;
  if (mode == 0 && c->opt.cascadic && c->nlev() > 1 && !(r0 <= tol_abs) && std::isfinite(r0)) {
    cascade(c);
    R.history[R.history_len++] = c->cur.rn;
  }
  double best = r0;
  while (true) {
    double rn = c->cur.rn;
    if (!std::isfinite(rn)) { st = NLMG_EDIVERGED; break; }
    if (rn <= tol_rel * r0 || rn <= tol_abs) break;
    if (cycles >= max_cycles) { st = NLMG_ENOCONV; break; }
    if (mode == 2) {
      newton_step(c);
    } else if (picard_only) {
      smooth0(c, 1);
    } else {
      early = vcycle(c, r0, tol_rel, tol_abs);
    }
    ++cycles;
    if (R.history_len < 64) R.history[R.history_len++] = c->cur.rn;
    // Inexact inner solves: once the iteration is in its asymptotic phase (residual below 1e-2 of the initial one),
    // a cycle that gains less than 10% on the best residual so far is taken as a sign that the loose inner
    // tolerances limit the outer progress, and both are divided by 100 (floor 1e-12) for the rest of the solve.
    if (best < 1e-2 * r0 && c->cur.rn > 0.9 * best &&
        (c->lin_tol_eff > 1e-12 || c->coarse_lin_tol_eff > 1e-12)) {
      c->lin_tol_eff = std::max(1e-12, c->lin_tol_eff * 1e-2);
      c->coarse_lin_tol_eff = std::max(1e-12, c->coarse_lin_tol_eff * 1e-2);
      c->coarsest_lin_tol_eff = std::max(1e-12, c->coarsest_lin_tol_eff * 1e-2);
      c->newton_tol_eff = std::max(1e-12, c->newton_tol_eff * 1e-2);
      c->tightenings++;
    }
    best = std::min(best, c->cur.rn);
    if (early) {
      if (!std::isfinite(c->cur.rn)) st = NLMG_EDIVERGED;
      break;
    }
  }
  c->opt.smoother = saved_smoother;
  CK(cudaMemcpyAsync(p_dev, c->cur.p, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaEventRecord(e1, c->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  R.cycles = cycles;
  R.early_exit = early ? 1 : 0;
  R.res = c->cur.rn;
  R.solve_ms = ms;
  R.fine_evals = c->fine_evals;
  R.lin_iters = c->lin_iters;
  R.kernel_launches = launch_count_thread() - launches0;
  for (int l = 0; l < 8; ++l) R.lin_iters_level[l] = c->lin_iters_level[l];
  R.tol_tightened = c->tightenings;
  R.newton_steps = (int32_t)c->newton_steps;
  c->prof_flush();
  if (rep) *rep = R;
  return st;
}

void need_device(nlmg_ctx* c) {
  if (!c->st) throw Error(NLMG_EINVAL, "context was built by nlmg_setup_host: no device data");
}

void need_data(nlmg_ctx* c) {
  need_device(c);
  if (!c->have_data) throw Error(NLMG_EINVAL, "call nlmg_set_data first");
}

}  // namespace

// ===================================================================================================================
// C ABI

extern "C" {

void nlmg_default_options(nlmg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_levels = 2;
  for (int l = 0; l < 8; ++l) {
    o->agg_size[l] = l == 0 ? 64 : 8;
    o->modes[l] = 4;
    o->flux_modes[l] = 1;
  }
  o->smoother = NLMG_SMOOTH_PICARD;
  o->nu_pre = o->nu_post = 2;
  o->omega = 0.8;
  o->bt_nmax = 4;
  o->bt_theta = 0.9;
  o->dp_clamp = 0.0;
  o->coarsest_steps = 10;
  o->coarsest_tol = 0.0;
  o->lin_tol = 1e-2;          // inner solves of the Picard smoothing steps: loose, the outer iteration corrects them
  o->lin_maxit = 5000;
  o->coarse_lin_tol = 1e-1;
  o->coarsest_lin_tol = 2e-1;
  o->lin_precision = 0;
  o->setup_threads = 0;
  o->newton_switch = 1e-3;
  o->newton_lin_tol = 1e-2;
  o->mg_row_cells = 16384;
}

static thread_local std::string g_setup_error;   // message of the calling thread's last failed setup

// The options a solve reads (those fixed at setup are checked there).
static bool solver_options_ok(const nlmg_options& o) {
  return (o.lin_precond == 0 || o.lin_precond == 1) && o.nu_pre >= 0 && o.nu_post >= 0 && o.bt_nmax >= 0 && o.omega > 0 && o.coarsest_steps >= 0 &&
         (o.lin_precision == 0 || o.lin_precision == 1 || o.lin_precision == 2) && o.max_sms >= 0 && o.smoother >= NLMG_SMOOTH_PICARD &&
         o.smoother <= NLMG_SMOOTH_PICARD_NEWTON && o.newton_switch >= 0.0 && o.newton_lin_tol > 0.0 &&
         (o.cascadic == 0 || o.cascadic == 1) && o.mg_row_cells >= 0;
}

static nlmg_status setup_impl(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt,
                              nlmg_ctx** out, bool device);

nlmg_status nlmg_setup(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt, nlmg_ctx** out) {
  return setup_impl(mesh, kappa, opt, out, true);
}

nlmg_status nlmg_setup_host(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt,
                            nlmg_ctx** out) {
  return setup_impl(mesh, kappa, opt, out, false);
}

// Stream-side state of one context: its stream (created by the caller), reduction scratch, barrier words, pinned
// read-back slots and every work buffer of the fine and coarse levels.
static void init_work(nlmg_ctx* c) {
  CK(cudaMallocHost(&c->h_sc, 16 * sizeof(double)));
  c->d_partial = c->dalloc<double>((size_t)2 * kPartStride);   // also the partials of the one-shot reductions
  c->d_cnt = c->dalloc<unsigned>(16);
  CK(cudaMemsetAsync(c->d_cnt, 0, 16 * sizeof(unsigned), c->st));
  c->d_sc = c->dalloc<double>(64);
  static_assert(sizeof(CoarseStepResult) <= 2 * sizeof(PcgResult), "result slots");
  c->d_res = c->dalloc<PcgResult>(3);   // the CG result, then the coarse-step result (two slots)
  c->d_bar = c->dalloc<unsigned>(64);   // count and generation on separate 128-byte lines
  CK(cudaMemsetAsync(c->d_bar, 0, 64 * sizeof(unsigned), c->st));
  CK(cudaMallocHost(&c->h_res, 3 * sizeof(PcgResult)));
  CK(cudaMemsetAsync(c->d_sc, 0, 64 * sizeof(double), c->st));
  c->reset_inner_tols();
  alloc_fine(c);
  alloc_mg(c);
  c->CB.resize(c->nlev());
  for (int l = 1; l < c->nlev(); ++l) alloc_level(c, l);
  CK(cudaStreamSynchronize(c->st));
}

static nlmg_status setup_impl(const nlmg_mesh* mesh, const nlmg_kappa* kappa, const nlmg_options* opt,
                              nlmg_ctx** out, bool device) {
  if (!out) return NLMG_EINVAL;
  *out = nullptr;
  if (!mesh || !kappa || !opt || mesh->n_cells <= 0 || mesh->n_faces < 0 || !mesh->cell_volume ||
      !mesh->face_cells || !mesh->half_trans || !mesh->face_bc || !mesh->face_area)
    return NLMG_EINVAL;
  if (opt->n_levels < 1 || opt->n_levels > 8 || (kappa->kind != 0 && kappa->kind != 1)) return NLMG_EINVAL;
  if (!solver_options_ok(*opt)) {
    g_setup_error = "bad solver option";
    return NLMG_EINVAL;
  }
  nlmg_ctx* c = new nlmg_ctx();
  nlmg_status s = guarded(c, [&]() -> nlmg_status {
    c->opt = *opt;
    c->kind = kappa->kind;
    c->a = kappa->a;
    FineMesh& fm = c->fm();
    fm.n_cells = mesh->n_cells;
    fm.n_faces = mesh->n_faces;
    fm.vol.assign(mesh->cell_volume, mesh->cell_volume + mesh->n_cells);
    fm.area.assign(mesh->face_area, mesh->face_area + mesh->n_faces);
    fm.bc.assign(mesh->face_bc, mesh->face_bc + mesh->n_faces);
    fm.fk.resize(mesh->n_faces);
    fm.fl.resize(mesh->n_faces);
    fm.ups0.resize(mesh->n_faces);
    fm.ups1.resize(mesh->n_faces);
    for (int f = 0; f < mesh->n_faces; ++f) {
      int K = mesh->face_cells[2 * f], L = mesh->face_cells[2 * f + 1];
      uint8_t b = fm.bc[f];
      if (b > 2 || K < 0 || K >= mesh->n_cells) throw Error(NLMG_EINVAL, "bad face " + std::to_string(f));
      if (b == 0 && (L <= K || L >= mesh->n_cells)) throw Error(NLMG_EINVAL, "interior face needs K < L");
      fm.fk[f] = K;
      fm.fl[f] = b == 0 ? L : -1;
      fm.ups0[f] = mesh->half_trans[2 * f];
      fm.ups1[f] = mesh->half_trans[2 * f + 1];
      if (b != 2 && !(fm.ups0[f] > 0)) throw Error(NLMG_EINVAL, "half transmissibility must be positive");
      if (b == 0 && !(fm.ups1[f] > 0)) throw Error(NLMG_EINVAL, "half transmissibility must be positive");
    }
    Options ho;
    ho.n_levels = opt->n_levels;
    for (int l = 0; l < 8; ++l) {
      ho.agg_size[l] = opt->agg_size[l];
      ho.modes[l] = opt->modes[l];
      ho.flux_modes[l] = opt->flux_modes[l];
      if (l + 1 < opt->n_levels && (opt->agg_size[l] < 2 || opt->modes[l] < 1 || opt->modes[l] > kMaxM))
        throw Error(NLMG_EINVAL, "agg_size >= 2 and 1 <= modes <= 8 per level");
      if (l + 1 < opt->n_levels && (opt->flux_modes[l] < 1 || opt->flux_modes[l] > 8))
        throw Error(NLMG_EINVAL, "1 <= flux_modes <= 8 per level");
    }
    ho.threads = opt->setup_threads;
    if (device) {
      ho.gpu_eig = true;
      ho.eig_fn = batched_smallest_eig;
    }
    // the multigrid preconditioner wants a coarsest level of at most kMgMaxCoarse pressure unknowns: coarsen further
    // (aggregates of agg_size[l] cells, the last FAS step's modes, one flux unknown per interface) for it alone
    if (opt->lin_precond == 1) {
      const int mlast = opt->n_levels >= 2 ? opt->modes[opt->n_levels - 2] : opt->modes[0];
      ho.n_levels = std::min(8, opt->n_levels + 4);
      for (int l = opt->n_levels - 1; l < 8; ++l) {
        if (l < 0) continue;
        if (ho.agg_size[l] < 2) ho.agg_size[l] = 8;
        ho.modes[l] = std::max(1, std::min(kMaxM, mlast));
        ho.flux_modes[l] = 1;
      }
    }
    std::string err;
    if (!build_hierarchy(fm, ho, c->H(), err)) throw Error(NLMG_EINVAL, err);
    Hierarchy& H = c->H();
    int mg_levels = 0;
    if (opt->lin_precond == 1) {
      mg_levels = mg_levels_for(H);
      if (mg_levels < 2)
        throw Error(NLMG_EUNSUPPORTED, "lin_precond = 1: no coarse level of at most " +
                                           std::to_string(kMgMaxCoarse) + " pressure unknowns within 8 levels");
      const int keep = std::max(opt->n_levels, mg_levels);
      H.levels.resize(keep);
      H.transfers.resize(keep - 1);
    }
    c->sh->n_fas = opt->n_levels;
    if (!device) return NLMG_OK;
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    upload_fine(c);
    c->LD.resize(c->nlev());
    c->TD.resize(std::max(0, c->nlev() - 1));
    for (int l = 1; l < c->nlev(); ++l) upload_level(c, l);
    for (int l = 0; l + 1 < c->nlev(); ++l) upload_transfer(c, l);
    if (mg_levels >= 2) upload_mg(c, mg_levels);
    c->sh->F = c->F;
    c->sh->LD = c->LD;
    c->sh->TD = c->TD;
    init_work(c);
    return NLMG_OK;
  });
  if (s != NLMG_OK) {
    g_setup_error = c->err;   // the context is freed: its message stays readable through nlmg_last_error(NULL)
    nlmg_destroy(c);
    return s;
  }
  *out = c;
  return NLMG_OK;
}

nlmg_status nlmg_instance(const nlmg_ctx* base, const nlmg_kappa* kappa, nlmg_ctx** out) {
  if (!out) return NLMG_EINVAL;
  *out = nullptr;
  if (!base || !base->st) return NLMG_EINVAL;
  if (kappa && kappa->kind != 0 && kappa->kind != 1) return NLMG_EINVAL;
  nlmg_ctx* c = new nlmg_ctx();
  nlmg_status s = guarded(c, [&]() -> nlmg_status {
    c->opt = base->opt;
    c->kind = kappa ? kappa->kind : base->kind;
    c->a = kappa ? kappa->a : base->a;
    c->sh = base->sh;
    c->F = c->sh->F;
    c->LD = c->sh->LD;
    c->TD = c->sh->TD;
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    init_work(c);
    return NLMG_OK;
  });
  if (s != NLMG_OK) {
    nlmg_destroy(c);
    return s;
  }
  *out = c;
  return NLMG_OK;
}

nlmg_status nlmg_tune_sm_share(nlmg_ctx* c, int32_t n_streams, const double* f_cell, const double* g_face,
                               int32_t* best_max_sms, double* solves_per_s) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (n_streams < 1 || !f_cell || !g_face || !best_max_sms) throw Error(NLMG_EINVAL, "bad argument");
    int sms = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // explicit SM counts: max_sms = 0 would mean the default share of nlmg_solve_many, not the whole GPU
    const int cand[4] = {sms, std::max(1, sms / 2), std::max(1, sms / 4), std::max(1, sms / 8)};
    const nlmg_options saved = c->opt;
    const size_t N = (size_t)c->F.N;
    std::vector<double> p(N * n_streams);
    std::vector<nlmg_report> rep(n_streams);
    std::vector<int32_t> st(n_streams);
    double best = -1.0;
    int best_i = 0;
    nlmg_status result = NLMG_OK;
    for (int i = 0; i < 4 && result == NLMG_OK; ++i) {
      c->opt.max_sms = cand[i];
      for (int run = 0; run < 2; ++run) {   // the first run is untimed (instances, caches)
        const auto t0 = std::chrono::steady_clock::now();
        const nlmg_status s = nlmg_solve_many(c, n_streams, f_cell, g_face, nullptr, c->tol_rel, c->tol_abs, 50,
                                              n_streams, p.data(), rep.data(), st.data());
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (s != NLMG_OK && s != NLMG_ENOCONV) {
          result = s;
          break;
        }
        if (run == 1) {
          const double v = n_streams / dt;
          if (solves_per_s) solves_per_s[i] = v;
          if (v > best) {
            best = v;
            best_i = i;
          }
        }
      }
    }
    c->opt = saved;
    c->reset_inner_tols();
    if (result != NLMG_OK) return result;
    *best_max_sms = cand[best_i];
    return NLMG_OK;
  });
}

nlmg_status nlmg_set_options(nlmg_ctx* c, const nlmg_options* opt) {
  return guarded(c, [&]() -> nlmg_status {
    if (!opt) throw Error(NLMG_EINVAL, "null options");
    if (opt->n_levels != c->opt.n_levels) throw Error(NLMG_EINVAL, "n_levels is fixed at setup");
    for (int l = 0; l + 1 < c->opt.n_levels; ++l)
      if (opt->agg_size[l] != c->opt.agg_size[l] || opt->modes[l] != c->opt.modes[l] ||
          opt->flux_modes[l] != c->opt.flux_modes[l])
        throw Error(NLMG_EINVAL, "agg_size, modes and flux_modes are fixed at setup");
    if (!solver_options_ok(*opt)) throw Error(NLMG_EINVAL, "bad solver option");
    if (opt->lin_precond == 1 && c->sh->MG.L == 0)
      throw Error(NLMG_EINVAL, "lin_precond = 1 needs a context set up with lin_precond = 1");
    const int threads = c->opt.setup_threads;
    c->opt = *opt;
    c->opt.setup_threads = threads;
    c->reset_inner_tols();
    c->newton_off = false;
    return NLMG_OK;
  });
}

static nlmg_status solve_many_impl(nlmg_ctx* c, int32_t n_rhs, const double* f_cell, const double* g_face,
                                   const double* x0, double tol_rel, double tol_abs, int32_t max_cycles,
                                   int32_t n_streams, double* p_out, nlmg_report* rep, int32_t* status, bool device) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (n_rhs < 0 || (n_rhs > 0 && (!f_cell || !g_face || !p_out))) throw Error(NLMG_EINVAL, "bad argument");
    if (n_rhs == 0) return NLMG_OK;
    const int ns = n_streams <= 0 ? 8 : n_streams;
    const int nw = std::max(1, std::min(ns, n_rhs));
    // The persistent kernels are latency bound, so contexts that run side by side do best on a share of the SMs
    // each: 1/min(n_streams, 4) of them (measured on the 64^3 workload: 4 streams on 38 SMs each 1.75x the
    // throughput of 4 streams on all SMs, 8 streams on 38 SMs each more again). The share follows from n_streams
    // alone, never from the load, so every row is reproducible bitwise (the reduction trees depend on the grid).
    int sms = 0, dev0 = 0;
    CK(cudaGetDevice(&dev0));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev0));
    const int share = ns > 1 ? std::max(1, sms / std::min(ns, 4)) : 0;
    std::vector<nlmg_ctx*> workers{c};
    {
      std::lock_guard<std::mutex> lk(c->pool_mu);
      while ((int)c->pool.size() < nw - 1) {
        nlmg_ctx* w = nullptr;
        nlmg_status st = nlmg_instance(c, nullptr, &w);
        if (st != NLMG_OK) throw Error(st, "creating a solve instance failed");
        c->pool.push_back(w);
      }
      for (int i = 0; i < nw - 1; ++i) {
        nlmg_ctx* w = c->pool[i];
        w->opt = c->opt;
        w->kind = c->kind;
        w->a = c->a;
        workers.push_back(w);
      }
    }
    for (nlmg_ctx* w : workers) w->auto_sm_cap = share;
    const size_t N = (size_t)c->F.N, NF = (size_t)c->fm().n_faces;
    std::vector<nlmg_status> st(n_rhs, NLMG_OK);
    std::vector<std::string> msg(n_rhs);
    std::atomic<int> next(0);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    auto run = [&](nlmg_ctx* w) {
      cudaSetDevice(dev);
      for (;;) {
        const int r = next.fetch_add(1);
        if (r >= n_rhs) break;
        st[r] = device ? nlmg_solve_device(w, f_cell + r * N, g_face + r * NF, x0 ? x0 + r * N : nullptr, tol_rel,
                                           tol_abs, max_cycles, p_out + r * N, rep ? rep + r : nullptr)
                       : nlmg_solve(w, f_cell + r * N, g_face + r * NF, x0 ? x0 + r * N : nullptr, tol_rel, tol_abs,
                                    max_cycles, p_out + r * N, rep ? rep + r : nullptr);
        if (st[r] != NLMG_OK) msg[r] = w->err;
      }
    };
    std::vector<std::thread> th;
    for (int i = 1; i < nw; ++i) th.emplace_back(run, workers[i]);
    run(c);
    for (auto& t : th) t.join();
    c->auto_sm_cap = 0;
    c->reset_inner_tols();
    nlmg_status worst = NLMG_OK;
    for (int r = 0; r < n_rhs; ++r) {
      if (status) status[r] = st[r];
      if (worst == NLMG_OK && st[r] != NLMG_OK) {
        worst = st[r];
        c->err = "right-hand side " + std::to_string(r) + ": " + msg[r];
      }
    }
    return worst;
  });
}

nlmg_status nlmg_solve_many(nlmg_ctx* c, int32_t n_rhs, const double* f_cell, const double* g_face,
                            const double* x0, double tol_rel, double tol_abs, int32_t max_cycles, int32_t n_streams,
                            double* p_out, nlmg_report* rep, int32_t* status) {
  return solve_many_impl(c, n_rhs, f_cell, g_face, x0, tol_rel, tol_abs, max_cycles, n_streams, p_out, rep, status,
                         false);
}

nlmg_status nlmg_solve_many_device(nlmg_ctx* c, int32_t n_rhs, const double* f_dev, const double* g_dev,
                                   const double* x0_dev, double tol_rel, double tol_abs, int32_t max_cycles,
                                   int32_t n_streams, double* p_dev, nlmg_report* rep, int32_t* status) {
  return solve_many_impl(c, n_rhs, f_dev, g_dev, x0_dev, tol_rel, tol_abs, max_cycles, n_streams, p_dev, rep, status,
                         true);
}

nlmg_status nlmg_set_data(nlmg_ctx* c, const double* f_cell, const double* g_face) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (!f_cell || !g_face) throw Error(NLMG_EINVAL, "null data");
    set_data_host(c, f_cell, g_face);
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_solve(nlmg_ctx* c, const double* f_cell, const double* g_face, const double* x0, double tol_rel,
                       double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (!f_cell || !g_face || !p_out) throw Error(NLMG_EINVAL, "null argument");
    set_data_host(c, f_cell, g_face);
    const double* x0d = nullptr;
    if (x0) {
      CK(cudaMemcpyAsync(c->fdp, x0, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
      x0d = c->fdp;
    }
    nlmg_status s = solve_core(c, x0d, tol_rel, tol_abs, max_cycles, c->fdp, rep, 0);
    CK(cudaMemcpyAsync(p_out, c->cur.p, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return s;
  });
}

nlmg_status nlmg_solve_device(nlmg_ctx* c, const double* f_dev, const double* g_dev, const double* x0_dev,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_dev, nlmg_report* rep) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (!f_dev || !g_dev || !p_dev) throw Error(NLMG_EINVAL, "null argument");
    set_data_dev(c, f_dev, g_dev);
    nlmg_status s = solve_core(c, x0_dev, tol_rel, tol_abs, max_cycles, p_dev, rep, 0);
    CK(cudaStreamSynchronize(c->st));
    return s;
  });
}

nlmg_status nlmg_solve_picard(nlmg_ctx* c, const double* f_cell, const double* g_face, const double* x0,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (!f_cell || !g_face || !p_out) throw Error(NLMG_EINVAL, "null argument");
    set_data_host(c, f_cell, g_face);
    const double* x0d = nullptr;
    if (x0) {
      CK(cudaMemcpyAsync(c->fdp, x0, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
      x0d = c->fdp;
    }
    nlmg_status s = solve_core(c, x0d, tol_rel, tol_abs, max_cycles, c->fdp, rep, 1);
    CK(cudaMemcpyAsync(p_out, c->cur.p, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return s;
  });
}


nlmg_status nlmg_solve_newton(nlmg_ctx* c, const double* f_cell, const double* g_face, const double* x0,
                              double tol_rel, double tol_abs, int32_t max_cycles, double* p_out, nlmg_report* rep) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (!f_cell || !g_face || !p_out) throw Error(NLMG_EINVAL, "null argument");
    set_data_host(c, f_cell, g_face);
    const double* x0d = nullptr;
    if (x0) {
      CK(cudaMemcpyAsync(c->fdp, x0, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
      x0d = c->fdp;
    }
    nlmg_status s = solve_core(c, x0d, tol_rel, tol_abs, max_cycles, c->fdp, rep, 2);
    CK(cudaMemcpyAsync(p_out, c->cur.p, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return s;
  });
}

nlmg_status nlmg_fine_residual(nlmg_ctx* c, const double* p, double* r_out) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    CK(cudaMemcpyAsync(c->cpa, p, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    fine_eval(c, c->cpa, nullptr, 0.0, c->t1);
    CK(cudaMemcpyAsync(r_out, c->t1.R, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_fine_flux(nlmg_ctx* c, const double* p, double* sigma_out) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    CK(cudaMemcpyAsync(c->cpa, p, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_kappa(c->st, c->F.N, c->cpa, nullptr, 0.0, c->cpa, c->t1.kap, nullptr, c->kind, c->a);
    launch_fine_flux(c->st, c->F, c->cpa, c->t1.kap, c->g, c->sig0);
    CK(cudaMemcpyAsync(sigma_out, c->sig0, (size_t)c->F.nflux * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_level_apply(nlmg_ctx* c, int32_t level, const double* x, double* out) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (level < 1 || level >= c->nlev()) throw Error(NLMG_EINVAL, "level must be a coarse level");
    const LevelDev& L = c->LD[level];
    CoarseBuf& B = c->CB[level];
    size_t nx = (size_t)L.nflux + L.np;
    CK(cudaMemcpyAsync(B.xt2, x, nx * sizeof(double), cudaMemcpyHostToDevice, c->st));
    coarse_res(c, level, B.xt2, nullptr, B.ptmp);
    CK(cudaMemcpyAsync(out, B.ptmp, nx * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_transfer(nlmg_ctx* c, int32_t level, int32_t op, const double* in, double* out) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (level < 0 || level + 1 >= c->nlev()) throw Error(NLMG_EINVAL, "no coarser level");
    const TransferDev& T = c->TD[level];
    const LevelDev& C = c->LD[level + 1];
    CoarseBuf& Bc = c->CB[level + 1];
    const size_t ncx = (size_t)C.nflux + C.np;
    size_t nfx;
    if (level == 0) nfx = c->F.N; else nfx = (size_t)c->LD[level].nflux + c->LD[level].np;
    const int nfs = level == 0 ? 0 : c->LD[level].nflux;   // flux length on the fine side
    double* fin = level == 0 ? c->cpa : c->CB[level].xt2;
    double* fout = level == 0 ? c->cpb : c->CB[level].ptmp;
    if (op == NLMG_PROJECT || op == NLMG_RESTRICT) {
      CK(cudaMemcpyAsync(fin, in, nfx * sizeof(double), cudaMemcpyHostToDevice, c->st));
      if (op == NLMG_PROJECT) {
        if (level == 0) {
          need_data(c);
          launch_kappa(c->st, c->F.N, fin, nullptr, 0.0, fin, c->t1.kap, nullptr, c->kind, c->a);
          launch_fine_flux(c->st, c->F, fin, c->t1.kap, c->g, c->sig0);
          launch_csr(c->st, T.qs_n, T.qs_off, T.qs_col, T.qs_val, c->sig0, Bc.xt2, 1.0, 0.0);
        } else {
          launch_csr(c->st, T.qs_n, T.qs_off, T.qs_col, T.qs_val, fin, Bc.xt2, 1.0, 0.0);
        }
      } else {
        if (level == 0)
          CK(cudaMemsetAsync(Bc.xt2, 0, C.nflux * sizeof(double), c->st));
        else
          launch_csr(c->st, T.pst_n, T.pst_off, T.pst_col, T.pst_val, fin, Bc.xt2, 1.0, 0.0);
      }
      launch_restrict_p(c->st, T, fin + nfs, Bc.xt2 + C.nflux, 1.0, nullptr, nullptr);
      CK(cudaMemcpyAsync(out, Bc.xt2, ncx * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    } else if (op == NLMG_PROLONG) {
      CK(cudaMemcpyAsync(Bc.xt2, in, ncx * sizeof(double), cudaMemcpyHostToDevice, c->st));
      if (level > 0) launch_csr(c->st, T.ps_n, T.ps_off, T.ps_col, T.ps_val, Bc.xt2, fout, 1.0, 0.0);
      launch_prolong_p(c->st, T, Bc.xt2 + C.nflux, fout + nfs);
      CK(cudaMemcpyAsync(out, fout, nfx * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    } else {
      throw Error(NLMG_EINVAL, "unknown transfer op");
    }
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_picard_update(nlmg_ctx* c, int32_t level, const double* x, const double* b, double* dx_out,
                               int32_t* iters) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (level < 0 || level >= c->nlev()) throw Error(NLMG_EINVAL, "bad level");
    c->reset_inner_tols();
    int it = 0;
    if (level == 0) {
      need_data(c);
      CK(cudaMemcpyAsync(c->cpa, x, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
      fine_eval(c, c->cpa, nullptr, 0.0, c->t1);
      launch_residual(c->st, c->F, c->t1.p, c->t1.kap, nullptr, c->g, c->rhs, c->t2.R, c->Tval, c->dinv, c->diagT,
                      nullptr, c->red(S_NORM2B));
      it = fine_pcg(c, c->t1.R, c->t1.kap);
      CK(cudaMemcpyAsync(dx_out, c->cx, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    } else {
      const LevelDev& L = c->LD[level];
      CoarseBuf& B = c->CB[level];
      size_t nx = (size_t)L.nflux + L.np;
      CK(cudaMemcpyAsync(B.x, x, nx * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(B.b, b, nx * sizeof(double), cudaMemcpyHostToDevice, c->st));
      // the fused coarse step the cycles run (one Picard step): its hybridized solve leaves the update in B.dx
      // (the clamp and Algorithm 1 after it only move x)
      const long long before = c->lin_iters_level[level];
      coarse_step(c, level, false, 1, level == c->nlev() - 1);
      it = (int)(c->lin_iters_level[level] - before);
      CK(cudaMemcpyAsync(dx_out, B.dx, nx * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    if (iters) *iters = it;
    return NLMG_OK;
  });
}

nlmg_status nlmg_precond_apply(nlmg_ctx* c, const double* p, const double* r, double* z_out) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    if (!p || !r || !z_out) throw Error(NLMG_EINVAL, "null argument");
    if (c->sh->MG.L == 0) throw Error(NLMG_EINVAL, "the context was not set up with lin_precond = 1");
    const MgDev& M = c->sh->MG;
    MgWork& W = c->mg;
    const size_t N = (size_t)c->F.N;
    CK(cudaMemcpyAsync(c->cpa, p, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    fine_eval(c, c->cpa, nullptr, 0.0, c->t1);
    launch_residual(c->st, c->F, c->t1.p, c->t1.kap, nullptr, c->g, c->rhs, c->t2.R, c->Tval, c->dinv, c->diagT,
                    nullptr, c->red(S_NORM2B));
    mg_select_precision(c);
    mg_enqueue_setup(c->st, M, c->F, W, c->Tval, c->diagT, c->t1.kap);
    CK(cudaMemcpyAsync(W.kb, r, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    if (!W.g_apply) CK(mg_capture_apply(c->st, M, c->F, W, &W.g_apply));
    CK(cudaGraphLaunch(W.g_apply, c->st));
    count_launch(2 + mg_vcycle_kernels(M));
    CK(cudaMemcpyAsync(z_out, W.kx, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NLMG_OK;
  });
}

nlmg_status nlmg_newton_update(nlmg_ctx* c, const double* p, double* dx_out, int32_t* iters) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    if (!p || !dx_out) throw Error(NLMG_EINVAL, "null argument");
    c->reset_inner_tols();
    CK(cudaMemcpyAsync(c->fdp, p, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    fine_eval(c, c->fdp, nullptr, 0.0, c->cur);
    newton_linearize(c);
    const int it = fine_bicgstab(c, c->cur.R);
    CK(cudaMemcpyAsync(dx_out, c->cx, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (iters) *iters = it;
    return NLMG_OK;
  });
}

nlmg_status nlmg_vcycle(nlmg_ctx* c, const double* p_in, double r0, double* p_out, double* res_out,
                        int32_t* early_exit) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    c->reset_inner_tols();
    CK(cudaMemcpyAsync(c->fdp, p_in, (size_t)c->F.N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    fine_eval(c, c->fdp, nullptr, 0.0, c->cur);
    c->tol_rel = 1e-8;
    c->tol_abs = 1e-10;
    c->r0_ref = r0;
    bool e = vcycle(c, r0, c->tol_rel, c->tol_abs);
    CK(cudaMemcpyAsync(p_out, c->cur.p, (size_t)c->F.N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (res_out) *res_out = c->cur.rn;
    if (early_exit) *early_exit = e ? 1 : 0;
    return NLMG_OK;
  });
}

nlmg_status nlmg_level_info_get(nlmg_ctx* c, int32_t level, nlmg_level_info* out) {
  return guarded(c, [&]() -> nlmg_status {
    if (level < 0 || level >= c->nlev() || !out) throw Error(NLMG_EINVAL, "bad level");
    const Level& L = c->H().levels[level];
    out->n_cells = L.n_cells;
    out->n_flux = L.n_flux;
    out->n_p = L.n_p();
    out->n_lambda = 0;
    out->eig_host = level > 0 ? c->H().transfers[level - 1].eig_host : 0;
    if (level > 0)
      for (int8_t k : L.fkind) out->n_lambda += (k == KIND_IFACE);
    return NLMG_OK;
  });
}

nlmg_status nlmg_get_aggregates(nlmg_ctx* c, int32_t level, int32_t* agg_of, int32_t* m_out) {
  return guarded(c, [&]() -> nlmg_status {
    if (level < 0 || level + 1 >= c->nlev()) throw Error(NLMG_EINVAL, "bad level");
    const Transfer& T = c->H().transfers[level];
    if (agg_of) std::copy(T.agg_of.begin(), T.agg_of.end(), agg_of);
    if (m_out) std::copy(c->H().levels[level + 1].m.begin(), c->H().levels[level + 1].m.end(), m_out);
    return NLMG_OK;
  });
}

nlmg_status nlmg_get_transfer_dense(nlmg_ctx* c, int32_t level, int32_t which, double* dense) {
  return guarded(c, [&]() -> nlmg_status {
    if (level < 0 || level + 1 >= c->nlev() || !dense) throw Error(NLMG_EINVAL, "bad level");
    const Level& L = c->H().levels[level];
    const Level& C = c->H().levels[level + 1];
    const Transfer& T = c->H().transfers[level];
    if (which == 0) {
      size_t nc = C.n_p();
      std::fill(dense, dense + (size_t)L.n_p() * nc, 0.0);
      for (int a = 0; a < C.n_cells; ++a) {
        int t = 0;
        for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
          int cc = T.agg_cells[k];
          for (int r = 0; r < L.m[cc]; ++r, ++t)
            for (int j = 0; j < C.m[a]; ++j)
              dense[(size_t)(L.p_off[cc] + r) * nc + C.p_off[a] + j] = T.Pblk[T.pblk_off[a] + (size_t)t * C.m[a] + j];
        }
      }
    } else {
      const Csr& M = which == 1 ? T.Ps : T.Qs;
      if (which != 1 && which != 2) throw Error(NLMG_EINVAL, "which");
      std::fill(dense, dense + (size_t)M.nrows * M.ncols, 0.0);
      for (int r = 0; r < M.nrows; ++r)
        for (int k = M.off[r]; k < M.off[r + 1]; ++k) dense[(size_t)r * M.ncols + M.col[k]] += M.val[k];
    }
    return NLMG_OK;
  });
}

nlmg_status nlmg_profile(nlmg_ctx* c, int32_t enable) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    c->prof_flush();
    if (enable && c->prof.ev.empty()) {
      c->prof.ev.resize(2 * 4096);
      c->prof.kid.resize(4096);
      for (auto& e : c->prof.ev) CK(cudaEventCreate(&e));
    }
    c->prof.on = enable != 0;
    for (int k = 0; k < 8; ++k) { c->prof.ms[k] = 0.0; c->prof.n[k] = 0; c->prof.bytes[k] = 0.0; c->prof.flops[k] = 0.0; }
    return NLMG_OK;
  });
}

nlmg_status nlmg_profile_read(nlmg_ctx* c, int32_t kernel, int64_t* launches, double* total_ms,
                              double* bytes_per_launch, double* flops_per_launch) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (kernel < 0 || kernel > 7) throw Error(NLMG_EINVAL, "kernel id");
    c->prof_flush();
    if (launches) *launches = c->prof.n[kernel];
    if (total_ms) *total_ms = c->prof.ms[kernel];
    // algorithmic bytes: every array the kernel streams, read or written once; gathered neighbour values are
    // counted once (they are the same vector); SELL padding is not counted
    const double N = c->F.N, nnz = (double)c->sh->nnz_real;
    double b = 0.0;
    if (kernel != 2) b = c->prof.n[kernel] ? c->prof.bytes[kernel] / c->prof.n[kernel] : 0.0;
    if (kernel == 2) b = 20.0 * nnz + 8.0 * N * 4;                          // nbr + 2 ups, q, kap, rhs, R
    if (bytes_per_launch) *bytes_per_launch = b;
    if (flops_per_launch) *flops_per_launch = c->prof.n[kernel] ? c->prof.flops[kernel] / c->prof.n[kernel] : 0.0;
    return NLMG_OK;
  });
}

nlmg_status nlmg_fine_residual_noalloc(nlmg_ctx* c, const double* p_dev, double* r_dev, double* norm2_dev,
                                       void* stream) {
  return guarded(c, [&]() -> nlmg_status {
    need_data(c);
    if (!p_dev || !r_dev || !norm2_dev) throw Error(NLMG_EINVAL, "null device pointer");
    if (c->F.N > kNoallocMaxCells)
      throw Error(NLMG_EINVAL, "nlmg_fine_residual_noalloc: mesh has " + std::to_string(c->F.N) +
                                   " cells, more than its fixed scratch holds (" + std::to_string(kNoallocMaxCells) +
                                   ")");
    void* scratch = nullptr;
    std::string err;
    if (!noalloc_scratch_address(&scratch, err)) throw Error(NLMG_ECUDA, err);
    // g and [f] are ready: nlmg_set_data synchronizes the context stream before it returns
    if (!noalloc_residual((cudaStream_t)stream, scratch, c->F, p_dev, c->g, c->rhs, r_dev, norm2_dev, c->kind, c->a,
                          err))
      throw Error(NLMG_ECUDA, err);
    return NLMG_OK;
  });
}

nlmg_status nlmg_device_bytes(const nlmg_ctx* c, size_t* shared_bytes, size_t* own_bytes) {
  if (!c) return NLMG_EINVAL;
  if (shared_bytes) *shared_bytes = c->sh->bytes;
  if (own_bytes) *own_bytes = c->own_bytes;
  return NLMG_OK;
}

nlmg_status nlmg_check_grid_barrier(nlmg_ctx* c, int32_t blocks, int32_t absent_block, int64_t spin_limit,
                                    int32_t* passed) {
  return guarded(c, [&]() -> nlmg_status {
    need_device(c);
    if (blocks < 1 || absent_block >= blocks || spin_limit < 1024 || spin_limit > (int64_t)1 << 26)
      throw Error(NLMG_EINVAL, "nlmg_check_grid_barrier: blocks >= 1, absent_block < blocks and a spin limit in "
                               "[1024, 2^26] are required");
    GridSync gs{c->d_bar, &c->d_res->err, c->sm_cap};
    CK(cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned), c->st));
    CK(cudaMemsetAsync(c->d_res, 0, sizeof(PcgResult), c->st));
    CK(launch_barrier_probe(c->st, gs, c->d_partial, blocks, absent_block, (unsigned long long)spin_limit,
                            &c->d_res->iters));
    count_launch(1);
    CK(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(PcgResult), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (passed) *passed = c->h_res->iters;
    if (c->h_res->err) {
      c->err = "grid barrier wait gave up";
      return NLMG_ETIMEOUT;
    }
    return NLMG_OK;
  });
}

nlmg_status nlmg_measure_fp64(double* gflops) {
  if (!gflops) return NLMG_EINVAL;
  try {
    return measure_fp64_peak(gflops) ? NLMG_OK : NLMG_ECUDA;
  } catch (...) {
    return NLMG_ECUDA;
  }
}

const char* nlmg_last_error(const nlmg_ctx* c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

void nlmg_destroy(nlmg_ctx* c) {
  if (!c) return;
  for (nlmg_ctx* w : c->pool) nlmg_destroy(w);
  if (c->st) cudaStreamSynchronize(c->st);
  for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->h_gh) cudaFreeHost(c->h_gh);
  if (c->mg.h_sc) cudaFreeHost(c->mg.h_sc);
  for (cudaGraphExec_t g : {c->mg.g_pcg[0], c->mg.g_pcg[1], c->mg.g_bicg[0], c->mg.g_bicg[1], c->mg.g_apply})
    if (g) cudaGraphExecDestroy(g);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

}  // extern "C"
