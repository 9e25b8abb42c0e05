// Device kernels of the FAS path (sm_103a, FP64). Every reduction is deterministic: each block reduces in a fixed
// shuffle/shared-memory tree, writes one partial, and the last block to finish sums the partials in block order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nlmg {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;
constexpr int kMaxLoc = 128;     // max local flux unknowns of a coarse cell
constexpr int kMaxM = 8;         // max pressure unknowns of a coarse cell

// device scalar slots
enum Scalar { S_RZ = 0, S_ALPHA, S_BETA, S_RR, S_RR0, S_PQ, S_NORM2, S_NORM2B, S_MAX, S_SCRATCH = 16 };

struct Reduce {
  double* partial;    // kMaxBlocks * 4
  unsigned* counter;  // one counter per reduction call site
  double* out;        // result slot(s)
};

// ---------------------------------------------------------------------------------------------------------------
// Fine level (reduced TPFA, Sec. 2.1)
struct FineDev {
  int N = 0, nnz = 0, nflux = 0, nslice = 0;
  // interior neighbours per cell in SELL-32 layout: slice s = cells 32 s .. 32 s + 31, width sell_w[s]; entry j of
  // cell K sits at sell_off[s] + 32 j + (K & 31). Padding entries point to the cell itself with Ups = (1, 0).
  int *sell_off = nullptr, *sell_w = nullptr, *nbr = nullptr;
  double *ups_s = nullptr, *ups_n = nullptr;       // own / neighbour half transmissibility per entry
  int *dir_off = nullptr, *dir_face = nullptr;     // Dirichlet faces per cell (CSR)
  double* dir_ups = nullptr;
  int *neu_off = nullptr, *neu_face = nullptr;     // Neumann faces per cell (CSR)
  double* neu_area = nullptr;
  double* vol = nullptr;
  int *fl_k = nullptr, *fl_l = nullptr, *fl_face = nullptr;   // level-0 flux unknowns
  double *fl_u0 = nullptr, *fl_u1 = nullptr;
};

// The nonlinearity: kind 0 kappa = exp(a p), kind 1 kappa = (1 + p^2)^-1 (Sec. 4 examples), and its derivative.
__device__ __forceinline__ double kappa_of(double p, int kind, double a) {
  return kind == 0 ? exp(a * p) : 1.0 / (1.0 + p * p);
}
// 1 / kappa(p) without a division: exp(-a p), or 1 + p^2.
__device__ __forceinline__ double inv_kappa_of(double p, int kind, double a) {
  return kind == 0 ? exp(-a * p) : fma(p, p, 1.0);
}
__device__ __forceinline__ double dkappa_of(double p, int kind, double a) {
  if (kind == 0) return a * exp(a * p);
  double t = 1.0 + p * p;
  return -2.0 * p / (t * t);
}

// Coarse level (mixed, cell-by-cell: Prop. 1)
struct LevelDev {
  int nc = 0, nflux = 0, np = 0, nlam = 0, nyl = 0, nif = 0;
  int *m = nullptr, *p_off = nullptr, *loc_off = nullptr, *loc = nullptr;
  int *mat_off = nullptr, *dmat_off = nullptr;
  double *Mloc = nullptr, *Dloc = nullptr, *w = nullptr;
  int *f_y0 = nullptr, *f_y1 = nullptr;            // per flux unknown: its slots in the per-cell buffer (-1)
  int* own0 = nullptr;                             // per local slot: 1 if this cell is the first owner
  int* sad_off = nullptr;                          // per cell: offset of (nl+m)^2 inverse local saddle
  double* Sinv = nullptr;
  int *if_off = nullptr, *if_slot = nullptr, *if_lam = nullptr;   // per cell: interface slots, their lambda
  double* if_sign = nullptr;
  int* hc_off = nullptr;                           // per cell: nif x nif block of C S_ss C^T (kappa = 1)
  double* Hc = nullptr;
  int *lam_y0 = nullptr, *lam_y1 = nullptr;        // per lambda: its two entries in the per-interface buffer
  int* if_cell = nullptr;                          // per interface slot: its cell
  int* slot_cell = nullptr;                        // per local flux slot: its cell
  int* p_cell = nullptr;                           // per pressure unknown: its cell
  // H over the lambdas as a SELL-32 matrix (for the memory-resident pipelined CG of large levels): per slice of 32
  // lambdas its width and first entry; per entry (slice-major, lane fastest) the column lambda and the Hc indices of
  // its contributions from the row lambda's first and second slot (-1: none); per lambda the cells of its two slots.
  // Entry (l, m) = kappa_c0 Hc[i0] + kappa_c1 Hc[i1].
  int hs_n = 0;
  int *hs_w = nullptr, *hs_off = nullptr, *hs_col = nullptr, *hs_i0 = nullptr, *hs_i1 = nullptr;
  int *lam_c0 = nullptr, *lam_c1 = nullptr;
};

// Transfer between level l and l+1
struct TransferDev {
  int na = 0, nrows = 0;
  int *rows_off = nullptr, *rows = nullptr;        // per aggregate: level-l pressure unknowns of its block rows
  int* pblk_off = nullptr;
  double* Pblk = nullptr;
  int *mc = nullptr, *pc_off = nullptr;            // coarse modes and pressure offsets
  int *pd_agg = nullptr, *pd_row = nullptr;        // per level-l pressure unknown: aggregate, block row
  int ps_n = 0, pst_n = 0, qs_n = 0;
  int *ps_off = nullptr, *ps_col = nullptr;   double* ps_val = nullptr;    // P_sigma rows (level-l flux)
  int *pst_off = nullptr, *pst_col = nullptr; double* pst_val = nullptr;   // P_sigma^T rows (coarse flux)
  int *qs_off = nullptr, *qs_col = nullptr;   double* qs_val = nullptr;    // Q_sigma rows (coarse flux)
};

inline int grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > kMaxBlocks) b = kMaxBlocks;
  return (int)b;
}

// number of kernels launched by this process through the launchers below
long long launch_count();          // whole process
long long launch_count_thread();   // issued by the calling host thread
void count_launch(int n);

// launchers (kernels.cu)
void launch_kappa(cudaStream_t st, int n, const double* p, const double* dp, double s, double* q, double* kap,
                  double* dkap, int kind, double a);
void launch_rhs(cudaStream_t st, const FineDev& F, const double* f, const double* g, double* rhs);
void launch_residual(cudaStream_t st, const FineDev& F, const double* q, const double* kap, const double* dkap,
                     const double* g, const double* rhs, double* R, double* Tval, double* dinv, double* diagT,
                     double* jdiag, Reduce red, double* Joff = nullptr);
void launch_jac_apply(cudaStream_t st, const FineDev& F, const double* jdiag, const double* Joff,
                      const double* dinv, const double* v, double* w);
void launch_mdot(cudaStream_t st, int n, int nk, const double* V, const double* w, double* partial,
                 unsigned* counter, double* h);
void launch_orth_update(cudaStream_t st, int n, int nk, const double* V, const double* h, double* w, Reduce red);
void launch_scale_vec(cudaStream_t st, int n, const double* x, double s, double* y);
void launch_jacobi_dinv(cudaStream_t st, int n, const double* jdiag, const double* diagT, double* out);
void launch_scale_jac(cudaStream_t st, const FineDev& F, const double* jdiag, const double* Joff,
                      const double* jdinv, double* Js, double* jd, double* sS);
void launch_gmres_combine(cudaStream_t st, int n, int nk, const double* V, const double* y, const double* dinv,
                          double* x);
void launch_jacobi_update(cudaStream_t st, int n, const double* q, const double* R, const double* jdiag,
                          const double* diagT, double omega, double* qnew);
void launch_max_abs(cudaStream_t st, int n, const double* x, Reduce red);
void launch_axpy(cudaStream_t st, int n, const double* x, double s, const double* dx, double* out);
void launch_sub(cudaStream_t st, int n, const double* y, const double* x, double* out);
void launch_fine_flux(cudaStream_t st, const FineDev& F, const double* p, const double* kap, const double* g,
                      double* sigma);
void launch_restrict_p(cudaStream_t st, const TransferDev& T, const double* in1, double* out1, double scale1,
                       const double* in2, double* out2);
void launch_prolong_p(cudaStream_t st, const TransferDev& T, const double* e, double* out);
void launch_csr(cudaStream_t st, int nrows, const int* off, const int* col, const double* val, const double* x,
                double* y, double alpha, double beta);
void launch_coarse_cell(cudaStream_t st, const LevelDev& L, const double* sig, const double* p, const double* bp,
                        double* yl, double* rp, double* kapc, int kind, double a, Reduce red);
void launch_sdiag(cudaStream_t st, int n, const double* diagT, double* sdiag);
// FP64 FMA throughput of the current device in GFLOP/s (an FMA counts 2), from a synthetic kernel
bool measure_fp64_peak(double* gflops);
template <class T>
void launch_scale_sell(cudaStream_t st, const FineDev& F, const double* Tval, const double* sdiag, T* Ts);
void launch_coarse_flux(cudaStream_t st, const LevelDev& L, const double* yl, const double* bs, double* rs,
                        Reduce red);
void launch_coarse_pbar_max(cudaStream_t st, const LevelDev& L, const double* dp, Reduce red);

}  // namespace nlmg
