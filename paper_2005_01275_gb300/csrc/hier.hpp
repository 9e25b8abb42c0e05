// Host-side multilevel hierarchy (built once by nlmg_setup, then uploaded to the device).
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace nlmg {

enum FluxKind : int8_t { KIND_IFACE = 0, KIND_BDRY = 1, KIND_BUBBLE = 2 };

// Sparse matrix in compressed rows.
struct Csr {
  int nrows = 0, ncols = 0;
  std::vector<int> off, col;
  std::vector<double> val;
};

// The fine mesh as given to nlmg_setup, plus derived per-cell adjacency.
struct FineMesh {
  int n_cells = 0, n_faces = 0;
  std::vector<double> vol, ups0, ups1, area;
  std::vector<int> fk, fl;        // face cells (fl = -1 on boundary)
  std::vector<uint8_t> bc;        // 0 interior, 1 Dirichlet, 2 Neumann
};

// One level in mixed, cell-by-cell form (Prop. 1): M(Pi~ p) = sum_c W_c^T Mloc_c W_c / kappa(w_c . p_c),
// D = sum_c rows_c Dloc_c W_c.
struct Level {
  int n_cells = 0, n_flux = 0;
  std::vector<int> m, p_off;                 // pressure unknowns per cell, prefix
  std::vector<int8_t> fkind;                 // per flux unknown
  std::vector<int> fown0, fown1;             // owner cells (fown1 = -1 unless interface)
  std::vector<int> loc_off, loc;             // per cell: sorted global flux ids
  std::vector<int> mat_off;                  // per cell: offset of n_loc^2 block in Mloc
  std::vector<double> Mloc;
  std::vector<int> dmat_off;                 // per cell: offset of m x n_loc block in Dloc
  std::vector<double> Dloc;
  std::vector<double> w;                     // Pi~ weights, indexed by p_off
  std::vector<double> vol, ones;             // cell volume; the vector 1^l over pressure unknowns
  std::vector<int> face_of_flux;             // level 0: face id of each flux unknown
  int n_p() const { return p_off.empty() ? 0 : p_off.back(); }
  int nloc(int c) const { return loc_off[c + 1] - loc_off[c]; }
};

// Transfer between level l and l+1.
struct Transfer {
  std::vector<int> agg_of;                   // level-l cell -> coarse cell
  std::vector<int> agg_off, agg_cells;       // cells of each aggregate (sorted)
  std::vector<int> pblk_off;                 // per aggregate: offset of its (rows x m_a) block, row-major
  std::vector<double> Pblk;
  Csr Ps;                                    // P_sigma, rows = level-l flux unknowns
  Csr PsT;                                   // P_sigma^T, rows = coarse flux unknowns
  Csr Qs;                                    // Q_sigma, rows = coarse flux unknowns
  std::vector<double> eig_gap;               // lambda_{m+1} - lambda_m per aggregate (diagnostic)
  int eig_host = 0;                          // GPU eigensolves redone on the host (non-finite GPU result)
};

// Batched eigensolver callback (nmat, aoff, n, k, A_all, vals, voff, vecs, err); vals has kEigStride per matrix.
constexpr int kEigStride = 9;
using EigBatchFn = std::function<bool(int, const std::vector<long long>&, const std::vector<int>&,
                                      const std::vector<int>&, std::vector<double>&, std::vector<double>&,
                                      std::vector<long long>&, std::vector<double>&, std::string&)>;

struct Options {
  bool gpu_eig = false;      // local eigenproblems on the GPU (batched) instead of the host
  EigBatchFn eig_fn;
  int n_levels = 2;
  int agg_size[8] = {16, 8, 8, 8, 8, 8, 8, 8};
  int modes[8] = {2, 2, 2, 2, 2, 2, 2, 2};
  int flux_modes[8] = {1, 1, 1, 1, 1, 1, 1, 1};   // m_f: flux unknowns per coarse interface at most
  int threads = 0;
};

struct Hierarchy {
  std::vector<Level> levels;
  std::vector<Transfer> transfers;
};

// Deterministic greedy aggregation (the rule documented with nlmg_setup).
std::vector<int> aggregate_graph(int n, const std::vector<int>& nb_off, const std::vector<int>& nb, int target);

Level make_level0(const FineMesh& fm, int threads = 1);
// Builds levels 1.. and the transfers; returns false and sets err on failure.
bool build_hierarchy(const FineMesh& fm, const Options& opt, Hierarchy& H, std::string& err);

}  // namespace nlmg
