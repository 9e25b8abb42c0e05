// Host-side construction of the spectral multilevel hierarchy (App. A-C of the paper), FP64.
//
// Per coarsening step l -> l+1 (m_f = 1 flux unknown per coarse interface):
//  * aggregates of the level-l cell graph by the deterministic greedy rule (stands in for METIS, Sec. 3.1);
//  * P_A: the m smallest eigenvectors of D_N M_N^-1 D_N^T on the extended aggregate N(A) at kappa = 1
//    (eq. local-eigenvalue-problem), restricted to A, with q_PV = 1^l|_A / ||1^l|_A|| projected out and the
//    remaining directions orthonormalised by an SVD, q_PV first (eqs. structure_pressure_interpolation,
//    definition_q_pv); singular values <= 1e-10 of the largest are dropped;
//  * one flux basis function per coarse interface F = (a, b): sigma from the local saddle on A_a U A_b with pressure
//    data -1/||1_a||^2 on a, +1/||1_b||^2 on b (eq. local_problem_to_define_sigma_pv); with m_f = 1 its
//    restriction to each aggregate is also the trace extension of eq. local_neumann_boundary_value_problem (the two
//    problems have the same unique flux), so the whole local solution is the basis function;
//  * one boundary basis function per aggregate owning Dirichlet unknowns: the local saddle on A with those unknowns
//    kept and pressure data -1/||1_A||^2;
//  * m_A - 1 bubbles per aggregate: the Neumann saddle on A with pressure data q (each NPV column);
//  * Q_sigma: interface / boundary coefficient = outflow of the aggregate through the interface divided by that of
//    the basis function; bubble coefficients = P_NPV^T (D sigma)|_A; D^{l+1} = P_p^T D^l P_sigma;
//  * static local matrices M_a^{l+1} = P_sigma,a^T M_A^l P_sigma,a (Prop. 1, App. C) and the Pi~ weights
//    w_a = |A|^-1 sum_{c in a} |c| w_c^T P_a[rows of c] (eq. pwc_projector, applied recursively).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <deque>
#include <functional>
#include <map>
#include <thread>

#include "dense.hpp"
#include "hier.hpp"

namespace nlmg {

namespace {

constexpr double kTraceDrop = 1e-8;   // m_f > 1: singular values kept of the projected unit-norm traces

void parallel_for(int n, int threads, const std::function<void(int, int, int)>& body) {
  // body(begin, end, worker) over contiguous chunks claimed dynamically; results must not depend on the order
  if (threads <= 1 || n < 2) {
    body(0, n, 0);
    return;
  }
  std::atomic<int> next(0);
  const int chunk = std::max(1, n / (threads * 8));
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t]() {
      for (;;) {
        int b = next.fetch_add(chunk);
        if (b >= n) break;
        body(b, std::min(n, b + chunk), t);
      }
    });
  for (auto& th : pool) th.join();
}

// Per-thread scratch: stamped membership and position maps so that sets can be built without clearing.
struct Scratch {
  std::vector<int> cell_stamp, flux_stamp, flux_pos;
  std::vector<int> trow, tcol;   // D's entries in assembly order (row, flux column, value)
  std::vector<double> tval;
  int token = 0;
  void init(int nc, int nf) {
    cell_stamp.assign(nc, 0);
    flux_stamp.assign(nf, 0);
    flux_pos.assign(nf, -1);
    token = 0;
  }
  int next() { return ++token; }
};

// A local mixed problem on a set of cells S with flux unknowns U (sorted).
struct LocalProblem {
  std::vector<int> cells, U, prow;   // prow[k] = first local pressure row of cells[k]
  int np = 0;
  bool mdiag = false;                // M is diagonal (level 0: TPFA): only Md and the sparse D are stored
  std::vector<double> M, Md, D, ones;   // M: |U| x |U| (when not diagonal), Md: its diagonal, D: np x |U| (dense,
                                        // when M is not diagonal)
  std::vector<int> dc_off, dc_row;      // when M is diagonal: the nonzeros of D by flux column, rows ascending
  std::vector<double> dc_val;
};

// X = M^-1 D^T (|U| x np): dense, or by rows of its nonzeros (columns ascending) when M is diagonal.
struct LocalX {
  bool sparse = false;
  std::vector<double> dense;
  std::vector<double> mfac;   // Cholesky factor of M (dense case; kept for solves with a flux right-hand side)
  std::vector<int> off, col;
  std::vector<double> val;
};

void assemble_local(const Level& L, const std::vector<int>& cells, const std::vector<int>& U, Scratch& sc,
                    LocalProblem& lp) {
  lp.cells = cells;
  lp.U = U;
  const int ns = (int)U.size();
  int tok = sc.next();
  for (int k = 0; k < ns; ++k) {
    sc.flux_stamp[U[k]] = tok;
    sc.flux_pos[U[k]] = k;
  }
  lp.prow.resize(cells.size());
  lp.np = 0;
  for (size_t k = 0; k < cells.size(); ++k) {
    lp.prow[k] = lp.np;
    lp.np += L.m[cells[k]];
  }
  // M is assembled densely only when some off-diagonal entry is nonzero (coarse levels); the TPFA level keeps its
  // diagonal alone, which saves the |U|^2 storage and scans that dominated the setup (same sums, same order)
  lp.Md.assign(ns, 0.0);
  lp.ones.assign(lp.np, 0.0);
  std::vector<int>& trow = sc.trow;
  std::vector<int>& tcol = sc.tcol;
  std::vector<double>& tval = sc.tval;
  trow.clear();
  tcol.clear();
  tval.clear();
  bool diag = true;
  for (size_t k = 0; k < cells.size(); ++k) {
    int c = cells[k];
    int nl = L.nloc(c), mc = L.m[c];
    const int* lc = &L.loc[L.loc_off[c]];
    const double* Mc = &L.Mloc[L.mat_off[c]];
    const double* Dc = &L.Dloc[L.dmat_off[c]];
    for (int r = 0; r < mc; ++r) lp.ones[lp.prow[k] + r] = L.ones[L.p_off[c] + r];
    for (int s = 0; s < nl; ++s) {
      if (sc.flux_stamp[lc[s]] != tok) continue;
      int ps = sc.flux_pos[lc[s]];
      for (int t = 0; t < nl; ++t) {
        if (sc.flux_stamp[lc[t]] != tok) continue;
        const int pt = sc.flux_pos[lc[t]];
        const double v = Mc[(size_t)s * nl + t];
        if (pt == ps)
          lp.Md[ps] += v;
        else if (v != 0.0)
          diag = false;
      }
      for (int r = 0; r < mc; ++r) {
        trow.push_back(lp.prow[k] + r);
        tcol.push_back(ps);
        tval.push_back(Dc[(size_t)r * nl + s]);
      }
    }
  }
  lp.mdiag = diag;
  lp.M.clear();
  lp.D.clear();
  lp.dc_off.clear();
  lp.dc_row.clear();
  lp.dc_val.clear();
  const size_t nt = trow.size();
  if (diag) {
    // D by flux column: a stable counting sort keeps each column's rows in generation order, which ascends (cells in
    // order, then their pressure rows); an entry met twice is summed in that order, as the dense assembly would
    lp.dc_off.assign(ns + 1, 0);
    for (size_t t = 0; t < nt; ++t) ++lp.dc_off[tcol[t] + 1];
    for (int i = 0; i < ns; ++i) lp.dc_off[i + 1] += lp.dc_off[i];
    std::vector<int> fill(lp.dc_off.begin(), lp.dc_off.end() - 1);
    lp.dc_row.assign(nt, 0);
    lp.dc_val.assign(nt, 0.0);
    for (size_t t = 0; t < nt; ++t) {
      const int at = fill[tcol[t]]++;
      lp.dc_row[at] = trow[t];
      lp.dc_val[at] = tval[t];
    }
    int w = 0;
    for (int i = 0; i < ns; ++i) {
      const int b = lp.dc_off[i], e = lp.dc_off[i + 1];
      lp.dc_off[i] = w;
      const int w0 = w;
      for (int t = b; t < e; ++t) {
        int hit = -1;
        for (int u = w0; u < w; ++u)
          if (lp.dc_row[u] == lp.dc_row[t]) hit = u;
        if (hit >= 0) {
          lp.dc_val[hit] += lp.dc_val[t];
        } else {
          lp.dc_row[w] = lp.dc_row[t];
          lp.dc_val[w] = lp.dc_val[t];
          ++w;
        }
      }
    }
    lp.dc_off[ns] = w;
    lp.dc_row.resize(w);
    lp.dc_val.resize(w);
    return;
  }
  lp.D.assign((size_t)lp.np * ns, 0.0);
  for (size_t t = 0; t < nt; ++t) lp.D[(size_t)trow[t] * ns + tcol[t]] += tval[t];
  lp.M.assign((size_t)ns * ns, 0.0);
  for (size_t k = 0; k < cells.size(); ++k) {
    int c = cells[k];
    int nl = L.nloc(c);
    const int* lc = &L.loc[L.loc_off[c]];
    const double* Mc = &L.Mloc[L.mat_off[c]];
    for (int s = 0; s < nl; ++s) {
      if (sc.flux_stamp[lc[s]] != tok) continue;
      int ps = sc.flux_pos[lc[s]];
      for (int t = 0; t < nl; ++t) {
        if (sc.flux_stamp[lc[t]] != tok) continue;
        lp.M[(size_t)ps * ns + sc.flux_pos[lc[t]]] += Mc[(size_t)s * nl + t];
      }
    }
  }
}

// Flux unknowns whose owners all lie in the stamped cell set: interfaces with both owners inside, bubbles.
std::vector<int> internal_flux(const Level& L, const std::vector<int>& cells, Scratch& sc) {
  int tok = sc.next();
  for (int c : cells) sc.cell_stamp[c] = tok;
  std::vector<int> U;
  for (int c : cells)
    for (int k = L.loc_off[c]; k < L.loc_off[c + 1]; ++k) {
      int i = L.loc[k];
      if (L.fkind[i] == KIND_IFACE) {
        if (sc.cell_stamp[L.fown0[i]] == tok && sc.cell_stamp[L.fown1[i]] == tok) U.push_back(i);
      } else if (L.fkind[i] == KIND_BUBBLE) {
        U.push_back(i);
      }
    }
  std::sort(U.begin(), U.end());
  U.erase(std::unique(U.begin(), U.end()), U.end());
  return U;
}

// Schur complement S = D M^-1 D^T and X = M^-1 D^T (|U| x np); returns false if M is not SPD. With a diagonal M both
// follow from D's nonzeros alone: every entry of S gathers the same products in the same order (flux columns
// ascending) as the dense form, whose other terms are zeros, so the result is the same to the bit.
bool schur(const LocalProblem& lp, std::vector<double>& S, LocalX& XL) {
  const int ns = (int)lp.U.size(), np = lp.np;
  XL.sparse = lp.mdiag;
  XL.dense.clear();
  XL.off.clear();
  XL.col.clear();
  XL.val.clear();
  if (lp.mdiag) {
    for (int i = 0; i < ns; ++i)
      if (!(lp.Md[i] > 0)) return false;
    XL.off = lp.dc_off;
    XL.col = lp.dc_row;
    XL.val.resize(lp.dc_val.size());
    for (int i = 0; i < ns; ++i)
      for (int t = lp.dc_off[i]; t < lp.dc_off[i + 1]; ++t) XL.val[t] = lp.dc_val[t] / lp.Md[i];
    S.assign((size_t)np * np, 0.0);
    for (int i = 0; i < ns; ++i)
      for (int t = lp.dc_off[i]; t < lp.dc_off[i + 1]; ++t) {
        const double d = lp.dc_val[t];
        if (d == 0.0) continue;
        double* Sr = &S[(size_t)lp.dc_row[t] * np];
        for (int u = lp.dc_off[i]; u < lp.dc_off[i + 1]; ++u) Sr[lp.dc_row[u]] += d * XL.val[u];
      }
    for (int r = 0; r < np; ++r)
      for (int q = r + 1; q < np; ++q) {
        double a = 0.5 * (S[(size_t)r * np + q] + S[(size_t)q * np + r]);
        S[(size_t)r * np + q] = S[(size_t)q * np + r] = a;
      }
    return true;
  }
  std::vector<double>& X = XL.dense;
  X.assign((size_t)ns * np, 0.0);
  {
    std::vector<double>& Lc = XL.mfac;
    Lc = lp.M;
    if (!chol_factor(ns, Lc.data())) return false;
    for (int r = 0; r < np; ++r)
      for (int i = 0; i < ns; ++i) X[(size_t)i * np + r] = lp.D[(size_t)r * ns + i];
    chol_solve_multi(ns, Lc.data(), np, X.data());
  }
  S.assign((size_t)np * np, 0.0);
  for (int r = 0; r < np; ++r) {
    const double* Dr = &lp.D[(size_t)r * ns];
    for (int i = 0; i < ns; ++i) {
      double d = Dr[i];
      if (d == 0.0) continue;
      const double* Xi = &X[(size_t)i * np];
      double* Sr = &S[(size_t)r * np];
      for (int q = 0; q < np; ++q) Sr[q] += d * Xi[q];
    }
  }
  for (int r = 0; r < np; ++r)
    for (int q = r + 1; q < np; ++q) {
      double a = 0.5 * (S[(size_t)r * np + q] + S[(size_t)q * np + r]);
      S[(size_t)r * np + q] = S[(size_t)q * np + r] = a;
    }
  return true;
}

// Factor for repeated local solves [M D^T; D 0][s; p] = [0; rp]. Without Dirichlet unknowns (a Neumann problem) S =
// D M^-1 D^T is singular with null space span(1^l) and rp is compatible (1^l . rp = 0); the pressure is then fixed by
// setting its unknown with the largest |1^l| entry to 0, which moves p along 1^l only and leaves s = -M^-1 D^T p
// unchanged (D^T 1^l = 0 on internal flux unknowns). S (or S without that row and column) is factored by Cholesky.
// The pinned row carries the rounding of the compatibility condition; one refinement step with the residual
// projected off 1^l leaves a residual along 1^l only, as a bordered solve would, so that P_NPV^T D s stays exact to
// rounding.
struct LocalSolver {
  const LocalProblem* lp = nullptr;
  LocalX X;                   // M^-1 D^T
  std::vector<double> U;      // upper Cholesky factor of the (reduced) S
  std::vector<double> S;      // the full S (Neumann problems, for the refinement step)
  int pin = -1;               // pressure unknown fixed to 0, or -1
  int nk = 0;
  bool init(const LocalProblem& p, bool neumann) {
    lp = &p;
    S.clear();
    if (!schur(p, S, X)) return false;
    const int np = p.np;
    pin = -1;
    if (neumann) {
      pin = 0;
      for (int r = 1; r < np; ++r)
        if (std::fabs(p.ones[r]) > std::fabs(p.ones[pin])) pin = r;
    }
    nk = np - (pin >= 0 ? 1 : 0);
    U.assign((size_t)nk * nk, 0.0);
    for (int r = 0, rr = 0; r < np; ++r) {
      if (r == pin) continue;
      for (int q = 0, qq = 0; q < np; ++q) {
        if (q == pin) continue;
        U[(size_t)rr * nk + qq] = S[(size_t)r * np + q];
        ++qq;
      }
      ++rr;
    }
    if (!neumann) std::vector<double>().swap(S);
    return chol_upper_factor(nk, U.data());
  }
  // S p = rhs with p[pin] = 0
  void pinned_solve(const std::vector<double>& rhs, std::vector<double>& pv) const {
    const int np = lp->np;
    std::vector<double> b(nk);
    for (int r = 0, rr = 0; r < np; ++r)
      if (r != pin) b[rr++] = rhs[r];
    chol_upper_solve(nk, U.data(), b.data());
    pv.assign(np, 0.0);
    for (int r = 0, rr = 0; r < np; ++r)
      if (r != pin) pv[r] = b[rr++];
  }
  // [M D^T; D 0][sigma; p] = [rs; rp]: y = M^-1 rs, S p = D y - rp, sigma = y - X p
  void solve_rhs(const std::vector<double>& rs, const std::vector<double>& rp, std::vector<double>& sigma) const {
    const int np = lp->np, ns = (int)lp->U.size();
    std::vector<double> y(rs), rq(rp);
    if (X.sparse) {
      for (int i = 0; i < ns; ++i) y[i] /= lp->Md[i];
      for (int i = 0; i < ns; ++i)
        for (int t = lp->dc_off[i]; t < lp->dc_off[i + 1]; ++t) rq[lp->dc_row[t]] -= lp->dc_val[t] * y[i];
    } else {
      chol_solve(ns, X.mfac.data(), y.data());
      for (int r = 0; r < np; ++r)
        for (int i = 0; i < ns; ++i) rq[r] -= lp->D[(size_t)r * ns + i] * y[i];
    }
    solve_p_rhs(rq, sigma);
    for (int i = 0; i < ns; ++i) sigma[i] += y[i];
  }
  // S p = -rp ; sigma = -X p
  void solve_p_rhs(const std::vector<double>& rp, std::vector<double>& sigma) const {
    const int np = lp->np, ns = (int)lp->U.size();
    std::vector<double> rhs(np), pv;
    for (int r = 0; r < np; ++r) rhs[r] = -rp[r];
    pinned_solve(rhs, pv);
    if (pin >= 0) {
      const std::vector<double>& one = lp->ones;
      double oo = 0.0, orr = 0.0;
      std::vector<double> res(np), dv;
      for (int r = 0; r < np; ++r) {
        double acc = rhs[r];
        const double* Sr = &S[(size_t)r * np];
        for (int q = 0; q < np; ++q) acc -= Sr[q] * pv[q];
        res[r] = acc;
        oo += one[r] * one[r];
        orr += one[r] * acc;
      }
      for (int r = 0; r < np; ++r) res[r] -= (orr / oo) * one[r];
      pinned_solve(res, dv);
      for (int r = 0; r < np; ++r) pv[r] += dv[r];
    }
    sigma.assign(ns, 0.0);
    for (int i = 0; i < ns; ++i) {
      double s = 0.0;
      if (X.sparse) {
        for (int t = X.off[i]; t < X.off[i + 1]; ++t) s += X.val[t] * pv[X.col[t]];
      } else {
        const double* Xi = &X.dense[(size_t)i * np];
        for (int r = 0; r < np; ++r) s += Xi[r] * pv[r];
      }
      sigma[i] = -s;
    }
  }
};

void sort_unique(std::vector<int>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

}  // namespace

std::vector<int> aggregate_graph(int n, const std::vector<int>& nb_off, const std::vector<int>& nb, int target) {
  std::vector<int> agg(n, -1);
  int nagg = 0;
  std::deque<int> q;
  for (int s = 0; s < n; ++s) {
    if (agg[s] != -1) continue;
    int id = nagg++;
    agg[s] = id;
    int count = 1;
    q.clear();
    q.push_back(s);
    while (!q.empty() && count < target) {
      int v = q.front();
      q.pop_front();
      for (int k = nb_off[v]; k < nb_off[v + 1]; ++k) {
        if (count >= target) break;
        int u = nb[k];
        if (agg[u] == -1) {
          agg[u] = id;
          ++count;
          q.push_back(u);
        }
      }
    }
  }
  // members per aggregate, kept current as merges happen
  std::vector<std::vector<int>> members(nagg);
  for (int v = 0; v < n; ++v) members[agg[v]].push_back(v);
  for (int id = 0; id < nagg; ++id) {
    auto& mem = members[id];
    if (mem.empty() || 2 * (long)mem.size() >= target) continue;
    std::map<int, int> shared;
    for (int v : mem)
      for (int k = nb_off[v]; k < nb_off[v + 1]; ++k) {
        int b = agg[nb[k]];
        if (b != id) shared[b] += 1;
      }
    if (shared.empty()) continue;
    int best = -1, bestc = -1;
    for (auto& kv : shared)                          // ascending id: first maximum wins ties
      if (kv.second > bestc) { bestc = kv.second; best = kv.first; }
    for (int v : mem) agg[v] = best;
    auto& dst = members[best];
    dst.insert(dst.end(), mem.begin(), mem.end());
    mem.clear();
  }
  std::vector<int> remap(nagg, -1);
  int next = 0;
  for (int id = 0; id < nagg; ++id)
    if (!members[id].empty()) remap[id] = next++;
  for (int v = 0; v < n; ++v) agg[v] = remap[agg[v]];
  return agg;
}

Level make_level0(const FineMesh& fm, int threads) {
  // Flux unknowns are the non-Neumann faces in face order, so appending each face's id to its owners' lists in face
  // order leaves every cell's list sorted; the lists are laid out by counting (no per-cell containers) and the local
  // matrices filled cell-parallel.
  Level L;
  const int n = fm.n_cells;
  L.n_cells = n;
  std::vector<int> cnt(n, 0);
  int nf = 0;
  for (int f = 0; f < fm.n_faces; ++f) {
    if (fm.bc[f] == 2) continue;
    ++nf;
    cnt[fm.fk[f]]++;
    if (fm.bc[f] == 0) cnt[fm.fl[f]]++;
  }
  L.n_flux = nf;
  L.face_of_flux.resize(nf);
  L.fkind.resize(nf);
  L.fown0.resize(nf);
  L.fown1.resize(nf);
  L.loc_off.assign(n + 1, 0);
  L.mat_off.assign(n + 1, 0);
  for (int c = 0; c < n; ++c) {
    L.loc_off[c + 1] = L.loc_off[c] + cnt[c];
    L.mat_off[c + 1] = L.mat_off[c] + cnt[c] * cnt[c];
  }
  L.dmat_off = L.loc_off;   // one pressure unknown per cell
  L.loc.resize(L.loc_off[n]);
  std::vector<int8_t> side(L.loc_off[n]);   // 0: the cell is the face's first owner
  {
    std::vector<int> fill(L.loc_off.begin(), L.loc_off.end() - 1);
    int j = 0;
    for (int f = 0; f < fm.n_faces; ++f) {
      if (fm.bc[f] == 2) continue;
      const bool itf = fm.bc[f] == 0;
      L.face_of_flux[j] = f;
      L.fkind[j] = itf ? KIND_IFACE : KIND_BDRY;
      L.fown0[j] = fm.fk[f];
      L.fown1[j] = itf ? fm.fl[f] : -1;
      L.loc[fill[fm.fk[f]]] = j;
      side[fill[fm.fk[f]]++] = 0;
      if (itf) {
        L.loc[fill[fm.fl[f]]] = j;
        side[fill[fm.fl[f]]++] = 1;
      }
      ++j;
    }
  }
  L.Mloc.assign((size_t)L.mat_off[n], 0.0);
  L.Dloc.assign((size_t)L.loc_off[n], 0.0);
  parallel_for(n, threads, [&](int b, int e, int) {
    for (int c = b; c < e; ++c) {
      const int k0 = L.loc_off[c], nl = L.loc_off[c + 1] - k0;
      const size_t mo = (size_t)L.mat_off[c];
      for (int s = 0; s < nl; ++s) {
        const int f = L.face_of_flux[L.loc[k0 + s]];
        const double ups = side[k0 + s] == 0 ? fm.ups0[f] : fm.ups1[f];
        L.Mloc[mo + (size_t)s * nl + s] = 1.0 / ups;
        L.Dloc[k0 + s] = side[k0 + s] == 0 ? -1.0 : 1.0;
      }
    }
  });
  L.m.assign(n, 1);
  L.p_off.resize(n + 1);
  for (int c = 0; c <= n; ++c) L.p_off[c] = c;
  L.w.assign(n, 1.0);
  L.vol = fm.vol;
  L.ones.assign(n, 1.0);
  return L;
}

// One coarsening step.
static bool coarsen(const Level& L, int target, int modes, int flux_modes, int threads, bool use_gpu_eig,
                    const EigBatchFn& eig_fn, Level& C, Transfer& T, std::string& err) {
  const int n = L.n_cells;
  // ---- cell graph ----------------------------------------------------------------------------------------------
  // adjacency lists by counting, then each list sorted and made unique (cell-parallel) and compacted
  std::vector<int> nb_off(n + 1, 0), nb;
  {
    std::vector<int> raw_off(n + 1, 0);
    for (int i = 0; i < L.n_flux; ++i)
      if (L.fkind[i] == KIND_IFACE) {
        raw_off[L.fown0[i] + 1]++;
        raw_off[L.fown1[i] + 1]++;
      }
    for (int v = 0; v < n; ++v) raw_off[v + 1] += raw_off[v];
    std::vector<int> raw(raw_off[n]), fill(raw_off.begin(), raw_off.end() - 1), len(n, 0);
    for (int i = 0; i < L.n_flux; ++i)
      if (L.fkind[i] == KIND_IFACE) {
        raw[fill[L.fown0[i]]++] = L.fown1[i];
        raw[fill[L.fown1[i]]++] = L.fown0[i];
      }
    parallel_for(n, threads, [&](int b, int e, int) {
      for (int v = b; v < e; ++v) {
        int* lo = raw.data() + raw_off[v];
        int* hi = raw.data() + raw_off[v + 1];
        std::sort(lo, hi);
        len[v] = (int)(std::unique(lo, hi) - lo);
      }
    });
    for (int v = 0; v < n; ++v) nb_off[v + 1] = nb_off[v] + len[v];
    nb.resize(nb_off[n]);
    parallel_for(n, threads, [&](int b, int e, int) {
      for (int v = b; v < e; ++v) std::copy(raw.begin() + raw_off[v], raw.begin() + raw_off[v] + len[v], nb.begin() + nb_off[v]);
    });
  }
  T.agg_of = aggregate_graph(n, nb_off, nb, target);
  int na = 0;
  for (int a : T.agg_of) na = std::max(na, a + 1);
  T.agg_off.assign(na + 1, 0);
  for (int v = 0; v < n; ++v) T.agg_off[T.agg_of[v] + 1]++;
  for (int a = 0; a < na; ++a) T.agg_off[a + 1] += T.agg_off[a];
  T.agg_cells.assign(n, 0);
  {
    std::vector<int> fill(T.agg_off.begin(), T.agg_off.end() - 1);
    for (int v = 0; v < n; ++v) T.agg_cells[fill[T.agg_of[v]]++] = v;
  }
  auto cells_of = [&](int a) { return std::vector<int>(&T.agg_cells[T.agg_off[a]], &T.agg_cells[T.agg_off[a + 1]]); };
  auto np_of = [&](int a) {
    int s = 0;
    for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) s += L.m[T.agg_cells[k]];
    return s;
  };
  std::vector<Scratch> scr(std::max(threads, 1));
  for (auto& s : scr) s.init(n, L.n_flux);
  // ---- spectral pressure bases ---------------------------------------------------------------------------------
  // pass 1: S_N = D_N M_N^-1 D_N^T on each extended aggregate; pass 2: its smallest eigenpairs (batched on the GPU
  // when available, else on the host); pass 3: restriction to A, q_PV first, SVD of the rest.
  std::vector<std::vector<double>> PA(na);
  std::vector<int> ma(na, 1);
  T.eig_gap.assign(na, 0.0);
  std::atomic<bool> fail(false);
  std::vector<std::vector<double>> Smat(na);
  std::vector<std::vector<int>> rows_in_N(na);
  std::vector<int> nS(na, 0), kS(na, 1);
  // m_f > 1: the rows of X_N = M_N^-1 D_N^T at the flux unknowns leaving A (one owner in A), restricted to A's
  // pressure rows, so that the traces of eq. definition-traces follow once P_A is known (CSR over A's rows)
  std::vector<std::vector<int>> xb_ids(na), xb_off(na), xb_col(na);
  std::vector<std::vector<double>> xb_val(na);
  parallel_for(na, threads, [&](int b, int e, int w) {
    Scratch& sc = scr[w];
    for (int a = b; a < e; ++a) {
      std::vector<int> cA = cells_of(a);
      std::vector<int> cN(cA);
      for (int c : cA) cN.insert(cN.end(), &nb[nb_off[c]], &nb[nb_off[c + 1]]);
      sort_unique(cN);
      std::vector<int> UN = internal_flux(L, cN, sc);
      LocalProblem lp;
      assemble_local(L, cN, UN, sc, lp);
      LocalX X;
      if (!schur(lp, Smat[a], X)) { fail = true; continue; }
      nS[a] = lp.np;
      kS[a] = std::min(modes, np_of(a));
      std::vector<int>& rows = rows_in_N[a];
      for (size_t k = 0, j = 0; k < cN.size(); ++k) {
        if (j < cA.size() && cN[k] == cA[j]) {
          for (int r = 0; r < L.m[cN[k]]; ++r) rows.push_back(lp.prow[k] + r);
          ++j;
        }
      }
      if (flux_modes > 1) {
        std::vector<int> tmap(lp.np, -1);
        for (size_t t = 0; t < rows.size(); ++t) tmap[rows[t]] = (int)t;
        auto inA = [&](int c) { return c >= 0 && std::binary_search(cA.begin(), cA.end(), c); };
        xb_off[a].push_back(0);
        for (size_t k = 0; k < UN.size(); ++k) {
          const int f = UN[k];
          if (L.fkind[f] != KIND_IFACE || inA(L.fown0[f]) == inA(L.fown1[f])) continue;
          xb_ids[a].push_back(f);
          if (X.sparse) {
            for (int t = X.off[k]; t < X.off[k + 1]; ++t)
              if (tmap[X.col[t]] >= 0) { xb_col[a].push_back(tmap[X.col[t]]); xb_val[a].push_back(X.val[t]); }
          } else {
            for (size_t t = 0; t < rows.size(); ++t) {
              const double v = X.dense[k * lp.np + rows[t]];
              if (v != 0.0) { xb_col[a].push_back((int)t); xb_val[a].push_back(v); }
            }
          }
          xb_off[a].push_back((int)xb_col[a].size());
        }
      }
    }
  });
  if (fail) { err = "local flux mass matrix not SPD in an eigenproblem"; return false; }
  std::vector<std::vector<double>> evecs(na);
  std::vector<double> evals_m(na), evals_next(na);
  bool done_gpu = false;
  if (use_gpu_eig && eig_fn) {
    std::vector<long long> aoff(na + 1, 0);
    for (int a = 0; a < na; ++a) aoff[a + 1] = aoff[a] + (long long)nS[a] * nS[a];
    std::vector<double> Aall(aoff[na]);
    for (int a = 0; a < na; ++a) std::copy(Smat[a].begin(), Smat[a].end(), Aall.begin() + aoff[a]);
    std::vector<double> vals, vecs;
    std::vector<long long> voff;
    std::string eerr;
    if (eig_fn(na, aoff, nS, kS, Aall, vals, voff, vecs, eerr)) {
      for (int a = 0; a < na; ++a) {
        evecs[a].assign(vecs.begin() + voff[a], vecs.begin() + voff[a + 1]);
        evals_m[a] = vals[(size_t)a * (kEigStride) + kS[a] - 1];
        evals_next[a] = vals[(size_t)a * (kEigStride) + kS[a]];
      }
      done_gpu = true;
    } else {
      err = eerr;
      return false;
    }
  }
  std::atomic<int> n_eig_host(0);
  parallel_for(na, threads, [&](int b, int e, int) {
    for (int a = b; a < e; ++a) {
      const int npA = np_of(a);
      const int m = kS[a];
      std::vector<double> vecs;
      bool gpu_ok = done_gpu && std::isfinite(evals_m[a]) && std::isfinite(evals_next[a]);
      if (gpu_ok)
        for (double v : evecs[a])
          if (!std::isfinite(v)) {
            gpu_ok = false;
            break;
          }
      if (gpu_ok) {
        vecs.swap(evecs[a]);
        T.eig_gap[a] = evals_next[a] - evals_m[a];
      } else {   // host path, also for a matrix whose batched GPU solve returned a non-finite value
        if (done_gpu) ++n_eig_host;
        std::vector<double> vals;
        double nextv = 0.0;
        sym_eig_smallest(nS[a], Smat[a], m, vals, vecs, &nextv);
        T.eig_gap[a] = nextv - vals[m - 1];
      }
      std::vector<double>().swap(Smat[a]);
      const std::vector<int>& rows = rows_in_N[a];
      std::vector<int> cA = cells_of(a);
      std::vector<double> q(npA);
      double qn = 0.0;
      {
        int t = 0;
        for (int c : cA)
          for (int r = 0; r < L.m[c]; ++r) { q[t] = L.ones[L.p_off[c] + r]; qn += q[t] * q[t]; ++t; }
      }
      qn = std::sqrt(qn);
      for (auto& x : q) x /= qn;
      std::vector<double> V((size_t)npA * m);
      for (int i = 0; i < npA; ++i)
        for (int jj = 0; jj < m; ++jj) V[(size_t)i * m + jj] = vecs[(size_t)rows[i] * m + jj];
      for (int jj = 0; jj < m; ++jj) {
        double dd = 0.0;
        for (int i = 0; i < npA; ++i) dd += q[i] * V[(size_t)i * m + jj];
        for (int i = 0; i < npA; ++i) V[(size_t)i * m + jj] -= dd * q[i];
      }
      std::vector<std::vector<double>> cols;
      cols.push_back(q);
      if (m > 1) {
        std::vector<double> U, sv;
        jacobi_svd(npA, m, V, U, sv);
        int keep = 0;
        if (sv[0] > 0)
          for (int jj = 0; jj < m; ++jj)
            if (sv[jj] > 1e-10 * sv[0]) keep++;
        keep = std::min(keep, std::min(m - 1, npA - 1));
        for (int jj = 0; jj < keep; ++jj) {
          std::vector<double> u(npA);
          int imax = 0;
          for (int i = 0; i < npA; ++i) {
            u[i] = U[(size_t)i * m + jj];
            if (std::fabs(u[i]) > std::fabs(u[imax])) imax = i;
          }
          if (u[imax] < 0)
            for (auto& x : u) x = -x;
          cols.push_back(u);
        }
      }
      ma[a] = (int)cols.size();
      PA[a].assign((size_t)npA * ma[a], 0.0);
      for (int i = 0; i < npA; ++i)
        for (int jj = 0; jj < ma[a]; ++jj) PA[a][(size_t)i * ma[a] + jj] = cols[jj][i];
    }
  });
  if (fail) { err = "local flux mass matrix not SPD in an eigenproblem"; return false; }
  T.eig_host = n_eig_host.load();
  T.pblk_off.assign(na + 1, 0);
  for (int a = 0; a < na; ++a) T.pblk_off[a + 1] = T.pblk_off[a] + (int)PA[a].size();
  T.Pblk.resize(T.pblk_off[na]);
  for (int a = 0; a < na; ++a) std::copy(PA[a].begin(), PA[a].end(), T.Pblk.begin() + T.pblk_off[a]);
  C.n_cells = na;
  C.m = ma;
  C.p_off.assign(na + 1, 0);
  for (int a = 0; a < na; ++a) C.p_off[a + 1] = C.p_off[a] + ma[a];
  C.ones.assign(C.p_off[na], 0.0);
  for (int a = 0; a < na; ++a) {
    int npA = np_of(a), t = 0;
    for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
      int c = T.agg_cells[k];
      for (int r = 0; r < L.m[c]; ++r, ++t)
        for (int j = 0; j < ma[a]; ++j)
          C.ones[C.p_off[a] + j] += PA[a][(size_t)t * ma[a] + j] * L.ones[L.p_off[c] + r];
    }
    (void)npA;
  }
  // ---- coarse interfaces, boundary sets ------------------------------------------------------------------------
  std::map<std::pair<int, int>, std::vector<int>> pairs;
  std::vector<std::vector<int>> bd(na);
  for (int i = 0; i < L.n_flux; ++i) {
    if (L.fkind[i] == KIND_IFACE) {
      int a = T.agg_of[L.fown0[i]], b = T.agg_of[L.fown1[i]];
      if (a != b) pairs[{std::min(a, b), std::max(a, b)}].push_back(i);
    } else if (L.fkind[i] == KIND_BDRY) {
      bd[T.agg_of[L.fown0[i]]].push_back(i);
    }
  }
  std::vector<std::pair<int, int>> plist;
  std::vector<std::vector<int>> Fdofs;
  for (auto& kv : pairs) {
    plist.push_back(kv.first);
    Fdofs.push_back(kv.second);
    sort_unique(Fdofs.back());
  }
  std::vector<int> bagg;
  for (int a = 0; a < na; ++a)
    if (!bd[a].empty()) bagg.push_back(a);
  const int nF = (int)plist.size(), nB = (int)bagg.size();
  std::vector<int> bub_off(na + 1, 0);
  for (int a = 0; a < na; ++a) bub_off[a + 1] = bub_off[a] + (ma[a] - 1);
  const int nC0 = nF + nB + bub_off[na];   // sigma^PV per interface, boundary unknowns, bubbles; m_f > 1 traces follow
  int nC = nC0;
  // basis functions as sparse columns (level-l flux id, value) and Q_sigma rows
  std::vector<std::vector<std::pair<int, double>>> psi(nC), qrow(nC);
  // m_f > 1: per interface the orthonormal traces kept beside sigma^PV and their Q_sigma rows (both on Fd)
  std::vector<std::vector<std::vector<double>>> extraU(nF), extraQ(nF);
  // outflow functional of aggregate a over a set of flux ids: t_i = -(1_a^T D)_i
  auto outflow_coef = [&](int a, const std::vector<int>& ids, Scratch& sc) {
    int tok = sc.next();
    for (int k = 0; k < (int)ids.size(); ++k) { sc.flux_stamp[ids[k]] = tok; sc.flux_pos[ids[k]] = k; }
    std::vector<double> t(ids.size(), 0.0);
    for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
      int c = T.agg_cells[k], nl = L.nloc(c);
      for (int s = 0; s < nl; ++s) {
        int i = L.loc[L.loc_off[c] + s];
        if (sc.flux_stamp[i] != tok) continue;
        double acc = 0.0;
        for (int r = 0; r < L.m[c]; ++r) acc += L.ones[L.p_off[c] + r] * L.Dloc[L.dmat_off[c] + (size_t)r * nl + s];
        t[sc.flux_pos[i]] -= acc;
      }
    }
    return t;
  };
  auto finish_trace = [&](int J, int a, const std::vector<int>& U, const std::vector<double>& sig,
                          const std::vector<int>& Fd, Scratch& sc) {
    for (size_t k = 0; k < U.size(); ++k) psi[J].push_back({U[k], sig[k]});
    std::vector<double> t = outflow_coef(a, Fd, sc);
    // value of the basis function on Fd
    double tot = 0.0;
    for (size_t k = 0; k < Fd.size(); ++k) {
      size_t pos = std::lower_bound(U.begin(), U.end(), Fd[k]) - U.begin();
      tot += t[k] * sig[pos];
    }
    for (size_t k = 0; k < Fd.size(); ++k) qrow[J].push_back({Fd[k], t[k] / tot});
    return tot != 0.0;
  };
  // m_f > 1 (eq. definition-traces, then an SVD): the traces (M_N^-1 D_N^T q_i)|_F from both aggregates' pressure
  // modes, each scaled to unit norm and projected by Pi_F = I - sigma^PV t^T / (t . sigma^PV) (t: outflow of a
  // through F), so that sigma^PV alone carries the net flux; the left singular vectors with value > 1e-8 are kept,
  // m_f - 1 and |F| - 1 at most, each with its first entry within 1e-6 of the largest magnitude positive; Q_sigma
  // row of a kept u: Pi_F^T u.
  auto interface_traces = [&](int J, int a, int bb, const std::vector<int>& U, const std::vector<double>& sig,
                              Scratch& sc) {
    const std::vector<int>& Fd = Fdofs[J];
    const int nf = (int)Fd.size();
    std::vector<double> t = outflow_coef(a, Fd, sc), sF(nf);
    double ts = 0.0;
    for (int k = 0; k < nf; ++k) {
      sF[k] = sig[std::lower_bound(U.begin(), U.end(), Fd[k]) - U.begin()];
      ts += t[k] * sF[k];
    }
    std::vector<std::vector<double>> tr;
    for (int side = 0; side < 2; ++side) {
      const int c = side ? bb : a;
      const std::vector<int>& ids = xb_ids[c];
      std::vector<int> rowk(nf);
      for (int k = 0; k < nf; ++k) {
        auto it = std::lower_bound(ids.begin(), ids.end(), Fd[k]);
        if (it == ids.end() || *it != Fd[k]) return false;
        rowk[k] = (int)(it - ids.begin());
      }
      for (int i = 0; i < ma[c]; ++i) {
        std::vector<double> v(nf, 0.0);
        double nv = 0.0;
        for (int k = 0; k < nf; ++k) {
          double acc = 0.0;
          for (int q = xb_off[c][rowk[k]]; q < xb_off[c][rowk[k] + 1]; ++q)
            acc += xb_val[c][q] * PA[c][(size_t)xb_col[c][q] * ma[c] + i];
          v[k] = acc;
          nv += acc * acc;
        }
        nv = std::sqrt(nv);
        if (nv > 0.0) {
          for (auto& x : v) x /= nv;
          tr.push_back(v);
        }
      }
    }
    if (tr.empty() || nf < 2) return true;
    const int m = (int)tr.size();
    std::vector<double> V((size_t)nf * m), Uu, sv;
    for (int j = 0; j < m; ++j) {
      double d = 0.0;
      for (int k = 0; k < nf; ++k) d += t[k] * tr[j][k];
      d /= ts;
      for (int k = 0; k < nf; ++k) V[(size_t)k * m + j] = tr[j][k] - sF[k] * d;
    }
    jacobi_svd(nf, m, V, Uu, sv);
    int keep = 0;
    for (int j = 0; j < m; ++j)
      if (sv[j] > kTraceDrop) keep++;
    keep = std::min(keep, std::min(flux_modes - 1, nf - 1));
    for (int j = 0; j < keep; ++j) {
      std::vector<double> u(nf);
      double umax = 0.0;
      for (int k = 0; k < nf; ++k) {
        u[k] = Uu[(size_t)k * m + j];
        umax = std::max(umax, std::fabs(u[k]));
      }
      int imax = 0;   // first entry within 1e-6 of the largest magnitude: mirror-symmetric ties do not pick the sign
      while (imax + 1 < nf && !(std::fabs(u[imax]) >= (1.0 - 1e-6) * umax)) ++imax;
      if (u[imax] < 0)
        for (auto& x : u) x = -x;
      double su = 0.0;
      for (int k = 0; k < nf; ++k) su += sF[k] * u[k];
      std::vector<double> qv(nf);
      for (int k = 0; k < nf; ++k) qv[k] = u[k] - t[k] * (su / ts);
      extraU[J].push_back(u);
      extraQ[J].push_back(qv);
    }
    return true;
  };
  parallel_for(nF, threads, [&](int b, int e, int w) {
    Scratch& sc = scr[w];
    for (int J = b; J < e; ++J) {
      int a = plist[J].first, bb = plist[J].second;
      std::vector<int> cU = cells_of(a), cb = cells_of(bb);
      cU.insert(cU.end(), cb.begin(), cb.end());
      sort_unique(cU);
      std::vector<int> U = internal_flux(L, cU, sc);
      LocalProblem lp;
      assemble_local(L, cU, U, sc, lp);
      LocalSolver ls;
      if (!ls.init(lp, true)) { fail = true; continue; }
      double na2 = 0.0, nb2 = 0.0;
      for (int c : cells_of(a))
        for (int r = 0; r < L.m[c]; ++r) na2 += L.ones[L.p_off[c] + r] * L.ones[L.p_off[c] + r];
      for (int c : cells_of(bb))
        for (int r = 0; r < L.m[c]; ++r) nb2 += L.ones[L.p_off[c] + r] * L.ones[L.p_off[c] + r];
      std::vector<double> rp(lp.np);
      for (size_t k = 0; k < cU.size(); ++k) {
        int c = cU[k];
        bool inA = T.agg_of[c] == a;
        for (int r = 0; r < L.m[c]; ++r)
          rp[lp.prow[k] + r] = (inA ? -1.0 / na2 : 1.0 / nb2) * L.ones[L.p_off[c] + r];
      }
      std::vector<double> sig;
      ls.solve_p_rhs(rp, sig);
      if (!finish_trace(J, a, U, sig, Fdofs[J], sc)) fail = true;
      if (flux_modes > 1 && !interface_traces(J, a, bb, U, sig, sc)) fail = true;
    }
  });
  parallel_for(nB, threads, [&](int b, int e, int w) {
    Scratch& sc = scr[w];
    for (int k = b; k < e; ++k) {
      int a = bagg[k], J = nF + k;
      std::vector<int> cA = cells_of(a);
      std::vector<int> U = internal_flux(L, cA, sc);
      std::vector<int> Bd = bd[a];
      sort_unique(Bd);
      U.insert(U.end(), Bd.begin(), Bd.end());
      sort_unique(U);
      LocalProblem lp;
      assemble_local(L, cA, U, sc, lp);
      LocalSolver ls;
      if (!ls.init(lp, false)) { fail = true; continue; }
      double n2 = 0.0;
      for (double x : lp.ones) n2 += x * x;
      std::vector<double> rp(lp.np);
      for (int r = 0; r < lp.np; ++r) rp[r] = -lp.ones[r] / n2;
      std::vector<double> sig;
      ls.solve_p_rhs(rp, sig);
      if (!finish_trace(J, a, U, sig, Bd, sc)) fail = true;
    }
  });
  parallel_for(na, threads, [&](int b, int e, int w) {
    Scratch& sc = scr[w];
    for (int a = b; a < e; ++a) {
      if (ma[a] <= 1) continue;
      std::vector<int> cA = cells_of(a);
      std::vector<int> U = internal_flux(L, cA, sc);
      LocalProblem lp;
      assemble_local(L, cA, U, sc, lp);
      LocalSolver ls;
      if (!ls.init(lp, true)) { fail = true; continue; }
      // (D sigma)|_A coefficients: for every flux id touching A, row r of Dloc scattered to global ids
      std::vector<int> touch;
      for (int c : cA) touch.insert(touch.end(), &L.loc[L.loc_off[c]], &L.loc[L.loc_off[c + 1]]);
      sort_unique(touch);
      for (int j = 1; j < ma[a]; ++j) {
        int J = nF + nB + bub_off[a] + (j - 1);
        std::vector<double> qj(lp.np);
        for (int r = 0; r < lp.np; ++r) qj[r] = PA[a][(size_t)r * ma[a] + j];
        std::vector<double> sig;
        ls.solve_p_rhs(qj, sig);                        // M sigma + D^T p = 0, D sigma = q_j
        for (size_t k = 0; k < U.size(); ++k) psi[J].push_back({U[k], sig[k]});
        std::vector<double> row(touch.size(), 0.0);
        for (size_t k = 0; k < cA.size(); ++k) {
          int c = cA[k], nl = L.nloc(c);
          for (int s = 0; s < nl; ++s) {
            int i = L.loc[L.loc_off[c] + s];
            size_t pos = std::lower_bound(touch.begin(), touch.end(), i) - touch.begin();
            double acc = 0.0;
            for (int r = 0; r < L.m[c]; ++r) acc += qj[lp.prow[k] + r] * L.Dloc[L.dmat_off[c] + (size_t)r * nl + s];
            row[pos] += acc;
          }
        }
        for (size_t k = 0; k < touch.size(); ++k)
          if (row[k] != 0.0) qrow[J].push_back({touch[k], row[k]});
      }
    }
  });
  if (fail) { err = "singular local problem while building the coarse flux space"; return false; }
  // m_f > 1: extend every kept trace u into both aggregates by the Neumann problem of App. A.2 (flux data
  // -M_{iF} u, pressure data c q - D_{AF} u with c = q . D_{AF} u), numbered after the bubbles, interface by interface
  std::vector<int> e_off(nF + 1, 0);
  for (int F = 0; F < nF; ++F) e_off[F + 1] = e_off[F] + (int)extraU[F].size();
  const int nE = e_off[nF];
  if (nE > 0) {
    std::vector<std::vector<int>> pairs_of(na);
    for (int F = 0; F < nF; ++F)
      if (!extraU[F].empty()) {
        pairs_of[plist[F].first].push_back(F);
        pairs_of[plist[F].second].push_back(F);
      }
    std::vector<std::vector<std::pair<int, double>>> extp((size_t)2 * nE);   // (trace, side) -> interior part
    parallel_for(na, threads, [&](int b, int e, int w) {
      Scratch& sc = scr[w];
      for (int a = b; a < e; ++a) {
        if (pairs_of[a].empty()) continue;
        std::vector<int> cA = cells_of(a);
        std::vector<int> U = internal_flux(L, cA, sc);
        if (U.empty()) continue;
        LocalProblem lp;
        assemble_local(L, cA, U, sc, lp);
        LocalSolver ls;
        if (!ls.init(lp, true)) { fail = true; continue; }
        double qn = 0.0;
        for (double x : lp.ones) qn += x * x;
        qn = std::sqrt(qn);
        for (int F : pairs_of[a]) {
          const int side = plist[F].first == a ? 0 : 1;
          const std::vector<int>& Fd = Fdofs[F];
          const int tok = sc.next();
          for (size_t k = 0; k < Fd.size(); ++k) {
            sc.flux_stamp[Fd[k]] = tok;
            sc.flux_pos[Fd[k]] = (int)k;
          }
          for (size_t j = 0; j < extraU[F].size(); ++j) {
            const std::vector<double>& u = extraU[F][j];
            std::vector<double> rs(U.size(), 0.0), dfu(lp.np, 0.0), rp(lp.np), sig;
            for (size_t kc = 0; kc < cA.size(); ++kc) {
              const int c = cA[kc], nl = L.nloc(c);
              const int* lc = &L.loc[L.loc_off[c]];
              const double* Mc = &L.Mloc[L.mat_off[c]];
              const double* Dc = &L.Dloc[L.dmat_off[c]];
              for (int tt = 0; tt < nl; ++tt) {
                if (sc.flux_stamp[lc[tt]] != tok) continue;
                const double ut = u[sc.flux_pos[lc[tt]]];
                for (int r = 0; r < L.m[c]; ++r) dfu[lp.prow[kc] + r] += Dc[(size_t)r * nl + tt] * ut;
                for (int ss = 0; ss < nl; ++ss) {
                  auto it = std::lower_bound(U.begin(), U.end(), lc[ss]);
                  if (it != U.end() && *it == lc[ss]) rs[it - U.begin()] -= Mc[(size_t)ss * nl + tt] * ut;
                }
              }
            }
            double cq = 0.0;
            for (int r = 0; r < lp.np; ++r) cq += lp.ones[r] / qn * dfu[r];
            for (int r = 0; r < lp.np; ++r) rp[r] = cq * lp.ones[r] / qn - dfu[r];
            ls.solve_rhs(rs, rp, sig);
            auto& dst = extp[(size_t)2 * (e_off[F] + j) + side];
            for (size_t k = 0; k < U.size(); ++k) dst.push_back({U[k], sig[k]});
          }
        }
      }
    });
    if (fail) { err = "singular local problem while extending the interface traces"; return false; }
    nC = nC0 + nE;
    psi.resize(nC);
    qrow.resize(nC);
    for (int F = 0; F < nF; ++F)
      for (size_t j = 0; j < extraU[F].size(); ++j) {
        const int i = e_off[F] + (int)j, J = nC0 + i;
        const std::vector<int>& Fd = Fdofs[F];
        psi[J] = extp[(size_t)2 * i];
        for (size_t k = 0; k < Fd.size(); ++k) psi[J].push_back({Fd[k], extraU[F][j][k]});
        psi[J].insert(psi[J].end(), extp[(size_t)2 * i + 1].begin(), extp[(size_t)2 * i + 1].end());
        for (size_t k = 0; k < Fd.size(); ++k) qrow[J].push_back({Fd[k], extraQ[F][j][k]});
      }
  }
  // ---- coarse level description ---------------------------------------------------------------------------------
  C.n_flux = nC;
  C.fkind.assign(nC, KIND_BUBBLE);
  C.fown0.assign(nC, -1);
  C.fown1.assign(nC, -1);
  for (int J = 0; J < nF; ++J) { C.fkind[J] = KIND_IFACE; C.fown0[J] = plist[J].first; C.fown1[J] = plist[J].second; }
  for (int k = 0; k < nB; ++k) { C.fkind[nF + k] = KIND_BDRY; C.fown0[nF + k] = bagg[k]; }
  for (int a = 0; a < na; ++a)
    for (int j = 1; j < ma[a]; ++j) C.fown0[nF + nB + bub_off[a] + j - 1] = a;
  for (int F = 0; F < nF; ++F)
    for (int i = e_off[F]; i < e_off[F + 1]; ++i) {
      C.fkind[nC0 + i] = KIND_IFACE;
      C.fown0[nC0 + i] = plist[F].first;
      C.fown1[nC0 + i] = plist[F].second;
    }
  std::vector<std::vector<int>> locs(na);
  for (int J = 0; J < nC; ++J) {
    locs[C.fown0[J]].push_back(J);
    if (C.fown1[J] >= 0) locs[C.fown1[J]].push_back(J);
  }
  C.loc_off.assign(na + 1, 0);
  for (int a = 0; a < na; ++a) {
    sort_unique(locs[a]);
    C.loc_off[a + 1] = C.loc_off[a] + (int)locs[a].size();
    C.loc.insert(C.loc.end(), locs[a].begin(), locs[a].end());
  }
  // P_sigma in both orientations and Q_sigma
  {
    parallel_for(nC, threads, [&](int b, int e, int) {
      for (int J = b; J < e; ++J) {
        std::sort(psi[J].begin(), psi[J].end());
        std::sort(qrow[J].begin(), qrow[J].end());
      }
    });
    T.PsT.nrows = nC;
    T.PsT.ncols = L.n_flux;
    T.PsT.off.assign(nC + 1, 0);
    T.Qs.nrows = nC;
    T.Qs.ncols = L.n_flux;
    T.Qs.off.assign(nC + 1, 0);
    for (int J = 0; J < nC; ++J) {
      T.PsT.off[J + 1] = T.PsT.off[J] + (int)psi[J].size();
      T.Qs.off[J + 1] = T.Qs.off[J] + (int)qrow[J].size();
    }
    T.PsT.col.resize(T.PsT.off[nC]);
    T.PsT.val.resize(T.PsT.off[nC]);
    T.Qs.col.resize(T.Qs.off[nC]);
    T.Qs.val.resize(T.Qs.off[nC]);
    parallel_for(nC, threads, [&](int b, int e, int) {
      for (int J = b; J < e; ++J) {
        int o = T.PsT.off[J];
        for (auto& x : psi[J]) { T.PsT.col[o] = x.first; T.PsT.val[o] = x.second; ++o; }
        o = T.Qs.off[J];
        for (auto& x : qrow[J]) { T.Qs.col[o] = x.first; T.Qs.val[o] = x.second; ++o; }
      }
    });
    // transpose: row i of P_sigma lists its coarse columns J in ascending order. Counted and filled in parallel
    // (relaxed atomic counters), then every row sorted by J: each (i, J) occurs once, so the layout does not depend on
    // the order the threads took
    T.Ps.nrows = L.n_flux;
    T.Ps.ncols = nC;
    T.Ps.off.assign(L.n_flux + 1, 0);
    {
      std::vector<int> cnt(L.n_flux, 0);
      parallel_for(nC, threads, [&](int b, int e, int) {
        for (int J = b; J < e; ++J)
          for (int q = T.PsT.off[J]; q < T.PsT.off[J + 1]; ++q)
            __atomic_fetch_add(&cnt[T.PsT.col[q]], 1, __ATOMIC_RELAXED);
      });
      for (int i = 0; i < L.n_flux; ++i) T.Ps.off[i + 1] = T.Ps.off[i] + cnt[i];
    }
    T.Ps.col.resize(T.PsT.col.size());
    T.Ps.val.resize(T.PsT.col.size());
    {
      std::vector<int> fill(T.Ps.off.begin(), T.Ps.off.end() - 1);
      parallel_for(nC, threads, [&](int b, int e, int) {
        for (int J = b; J < e; ++J)
          for (int q = T.PsT.off[J]; q < T.PsT.off[J + 1]; ++q) {
            const int pos = __atomic_fetch_add(&fill[T.PsT.col[q]], 1, __ATOMIC_RELAXED);
            T.Ps.col[pos] = J;
            T.Ps.val[pos] = T.PsT.val[q];
          }
      });
    }
    parallel_for(L.n_flux, threads, [&](int b, int e, int) {
      for (int i = b; i < e; ++i)   // insertion sort of the row by column (rows hold a few tens of entries)
        for (int k = T.Ps.off[i] + 1; k < T.Ps.off[i + 1]; ++k) {
          const int cj = T.Ps.col[k];
          const double vj = T.Ps.val[k];
          int t = k - 1;
          for (; t >= T.Ps.off[i] && T.Ps.col[t] > cj; --t) {
            T.Ps.col[t + 1] = T.Ps.col[t];
            T.Ps.val[t + 1] = T.Ps.val[t];
          }
          T.Ps.col[t + 1] = cj;
          T.Ps.val[t + 1] = vj;
        }
    });
  }
  // static local matrices, divergence blocks, Pi~ weights
  C.mat_off.assign(na + 1, 0);
  C.dmat_off.assign(na + 1, 0);
  for (int a = 0; a < na; ++a) {
    int nl = C.loc_off[a + 1] - C.loc_off[a];
    C.mat_off[a + 1] = C.mat_off[a] + nl * nl;
    C.dmat_off[a + 1] = C.dmat_off[a] + ma[a] * nl;
  }
  C.Mloc.assign(C.mat_off[na], 0.0);
  C.Dloc.assign(C.dmat_off[na], 0.0);
  C.w.assign(C.p_off[na], 0.0);
  C.vol.assign(na, 0.0);
  parallel_for(na, threads, [&](int b, int e, int) {
    for (int a = b; a < e; ++a) {
      int nl = C.loc_off[a + 1] - C.loc_off[a];
      const int* la = &C.loc[C.loc_off[a]];
      double vol = 0.0;
      for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) vol += L.vol[T.agg_cells[k]];
      C.vol[a] = vol;
      int t = 0;  // running row of P_a
      for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
        int c = T.agg_cells[k], nlc = L.nloc(c), mc = L.m[c];
        const int* lc = &L.loc[L.loc_off[c]];
        // Pc = P_sigma[loc_c, loc_a] (nlc x nl)
        std::vector<double> Pc((size_t)nlc * nl, 0.0);
        for (int s = 0; s < nlc; ++s) {
          int i = lc[s];
          for (int q = T.Ps.off[i]; q < T.Ps.off[i + 1]; ++q) {
            const int* pos = std::lower_bound(la, la + nl, T.Ps.col[q]);
            if (pos != la + nl && *pos == T.Ps.col[q]) Pc[(size_t)s * nl + (pos - la)] += T.Ps.val[q];
          }
        }
        const double* Mc = &L.Mloc[L.mat_off[c]];
        std::vector<double> MP((size_t)nlc * nl, 0.0);
        for (int s = 0; s < nlc; ++s)
          for (int u = 0; u < nlc; ++u) {
            double mv = Mc[(size_t)s * nlc + u];
            if (mv == 0.0) continue;
            for (int j = 0; j < nl; ++j) MP[(size_t)s * nl + j] += mv * Pc[(size_t)u * nl + j];
          }
        for (int s = 0; s < nlc; ++s)
          for (int i = 0; i < nl; ++i) {
            double ps = Pc[(size_t)s * nl + i];
            if (ps == 0.0) continue;
            for (int j = 0; j < nl; ++j) C.Mloc[C.mat_off[a] + (size_t)i * nl + j] += ps * MP[(size_t)s * nl + j];
          }
        // Dloc_a += P_a[rows_c]^T Dloc_c Pc
        const double* Dc = &L.Dloc[L.dmat_off[c]];
        std::vector<double> DP((size_t)mc * nl, 0.0);
        for (int r = 0; r < mc; ++r)
          for (int s = 0; s < nlc; ++s) {
            double dv = Dc[(size_t)r * nlc + s];
            if (dv == 0.0) continue;
            for (int j = 0; j < nl; ++j) DP[(size_t)r * nl + j] += dv * Pc[(size_t)s * nl + j];
          }
        for (int r = 0; r < mc; ++r) {
          const double* Prow = &T.Pblk[T.pblk_off[a] + (size_t)(t + r) * ma[a]];
          for (int i = 0; i < ma[a]; ++i)
            for (int j = 0; j < nl; ++j) C.Dloc[C.dmat_off[a] + (size_t)i * nl + j] += Prow[i] * DP[(size_t)r * nl + j];
          double wcr = L.w[L.p_off[c] + r] * L.vol[c];
          for (int i = 0; i < ma[a]; ++i) C.w[C.p_off[a] + i] += wcr * Prow[i];
        }
        t += mc;
      }
      for (int i = 0; i < ma[a]; ++i) C.w[C.p_off[a] + i] /= vol;
    }
  });
  return true;
}

// Every stored value of the hierarchy must be finite; returns false with the level and array otherwise.
static bool check_finite(const Hierarchy& H, std::string& err) {
  auto bad = [](const std::vector<double>& v) {
    for (double x : v)
      if (!std::isfinite(x)) return true;
    return false;
  };
  for (size_t l = 0; l < H.levels.size(); ++l) {
    const Level& L = H.levels[l];
    const char* what = bad(L.Mloc) ? "Mloc" : bad(L.Dloc) ? "Dloc" : bad(L.w) ? "Pi~ weights" : nullptr;
    if (what) {
      err = "non-finite value in the hierarchy: level " + std::to_string(l) + " " + what;
      return false;
    }
  }
  for (size_t l = 0; l < H.transfers.size(); ++l) {
    const Transfer& T = H.transfers[l];
    const char* what = bad(T.Pblk) ? "P_p" : bad(T.Ps.val) ? "P_sigma" : bad(T.Qs.val) ? "Q_sigma" : nullptr;
    if (what) {
      err = "non-finite value in the hierarchy: transfer " + std::to_string(l) + " " + what;
      return false;
    }
  }
  return true;
}

bool build_hierarchy(const FineMesh& fm, const Options& opt, Hierarchy& H, std::string& err) {
  int threads = opt.threads > 0 ? opt.threads : (int)std::max(1u, std::thread::hardware_concurrency());
  H.levels.clear();
  H.transfers.clear();
  H.levels.push_back(make_level0(fm, threads));
  for (int l = 0; l + 1 < opt.n_levels; ++l) {
    Level C;
    Transfer T;
    if (!coarsen(H.levels.back(), opt.agg_size[l], opt.modes[l], opt.flux_modes[l], threads, opt.gpu_eig,
                 opt.eig_fn, C, T, err))
      return false;
    H.levels.push_back(std::move(C));
    H.transfers.push_back(std::move(T));
  }
  return check_finite(H, err);
}

}  // namespace nlmg
