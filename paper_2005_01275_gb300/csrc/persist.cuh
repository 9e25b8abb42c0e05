// Persistent cooperative CG kernels (persist.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nlmg {

struct PcgResult {
  int iters;      // CG iterations taken
  int err;        // 1 if a grid barrier gave up waiting
  double rr0;     // ||r_0||^2
  double rr;      // ||r_final||^2
};

// The persistent kernels' reductions use two buffers of kPartStride per-block partial sums (>= blocks x values).
constexpr int kPartStride = 8192;

struct GridSync {
  unsigned* count;   // barrier arrival counter (0 at launch); own 128-byte line
  int* err;          // set when a wait gives up
  int sm_cap;        // host side: at most this many SMs for the launch (0 = all)
};

template <class T>
cudaError_t launch_fine_cg(cudaStream_t st, const FineDev& F, const T* Ts, const double* sdiag, const double* b,
                           double bscale, double* dx, T* y, T* r, T* pa, T* pb, T* q, double* partial, GridSync gs,
                           double tol, int maxit, PcgResult* res);

template <class T>
cudaError_t launch_fine_cg_pipe(cudaStream_t st, const FineDev& F, const T* Ts, const double* sdiag, const double* b,
                                double bscale, double* dx, T* y, T* r, T* wa, T* wb, T* z, T* sv, T* p,
                                double* partial, GridSync gs, double tol, int maxit, PcgResult* res);

// Register-resident pipelined CG (TM = type of the matrix and of the exchanged vector, double; recurrences in FP64).
// Returns cudaErrorNotSupported without launching when a thread would have to hold more than 4 cells.
template <class TM>
cudaError_t launch_fine_cg_reg(cudaStream_t st, const FineDev& F, const TM* Ts, const double* sdiag, const double* b,
                               double bscale, double* dx, TM* wa, TM* wb, double* partial, GridSync gs, double tol,
                               int maxit, PcgResult* res);

// Register-resident FP32 pipelined CG with residual replacement every `replace` iterations (0: never). Returns
// cudaErrorNotSupported without launching when a thread would have to hold more than 8 cells.
cudaError_t launch_fine_cg_rr32(cudaStream_t st, const FineDev& F, const float* Ts, const double* sdiag,
                                const double* b, double bscale, double* dx, float* wa, float* wb, float* ypub,
                                float* ppub, float* rpub, float* spub, double* partial, GridSync gs, double tol,
                                int maxit, int replace, PcgResult* res);

// Persistent FP64 BiCGStab for the level-0 Newton system J dx = bscale b on the scaled Jacobian (Js off the
// diagonal in the SELL layout, jd on it, sS = S per cell); work holds 7 n_cells doubles.
cudaError_t launch_fine_bicgstab(cudaStream_t st, const FineDev& F, const double* Js, const double* jd,
                                 const double* sS, const double* b, double bscale, double* dx, double* work,
                                 double* partial, GridSync gs, double tol, int maxit, PcgResult* res);

// Extra per-lambda vectors of the pipelined hybridized CG (w = H u, z, s, and m = M w double-buffered).
template <class T>
struct HybPipeBufs {
  T *w = nullptr, *z = nullptr, *s = nullptr, *ma = nullptr, *mb = nullptr;
};

// The linear parts of the coarse operator at a vector v = [sigma; p] with kappa left out: per local flux slot y of
// cell c (local index u) ms[y] = (M_c sigma_c)_u and ds[y] = (D_c^T p_c)_u (nyl each), per pressure unknown
// dr[i] = (D_c sigma_c)_i (np), per cell pb[c] = (Pi~ p)_c (nc).
struct LinParts {
  double *ms, *ds, *dr, *pb;
};

// Device buffers of one coarse level used by the fused Picard step (all of length nflux + np unless noted).
template <class T>
struct CoarseStepBufs {
  double *x, *b, *r, *nb, *dx;                    // iterate, rhs, residual, -residual, step
  double* kapc;                                   // kappa per cell (nc)
  LinParts base, dir;                             // linear parts at x and along dx (Algorithm 1's trials)
  T *ylam, *ydiag, *lam, *lr, *lz, *pa, *pb, *lq, *ldinv;   // hybridized CG (nif / nlam)
  HybPipeBufs<T> pipe;   // set: pipelined hybridized CG (one grid synchronisation per iteration)
  T* hsv = nullptr;      // L.hs_n values of the assembled H (memory-resident pipelined CG), or null
};

struct CoarseStepParams {
  int kind;
  double a;
  double dp_clamp;       // <= 0: off
  int bt_nmax;
  double bt_theta;
  int backtrack_first;   // 1: first x <- Algorithm 1 along the given dx from s = 1 (rn_in = ||r(x)||)
  double rn_in;
  int nsteps;            // Picard steps after that
  int coarsest;          // 1: stop the steps once ||r|| <= tol_rel ||r(x_entry)|| or ||r|| <= tol_abs
  double tol_rel, tol_abs;
  double lin_tol;
  int maxit;
};

struct CoarseStepResult {
  double rn;        // ||A(x) - b|| at the final x
  int iters;        // hybridized CG iterations
  int steps;        // Picard steps taken
  int res_evals;    // evaluations of the operator's linear parts (one per Picard step and one on entry)
  int bad;          // 0, or where a non-finite value appeared: 1 residual, 2 hybridized CG
  int trials;       // residual norms of Algorithm 1's trial points (from the linear parts)
};

// One launch: [Algorithm 1 along a given correction], up to nsteps coarse Picard steps (frozen-kappa hybridized
// solve, clamp on Pi~ dp, Algorithm 1), leaving the residual r = A(x) - b (and -r, kappa per cell) at the final x;
// every decision is taken on the device. The hybridized CG runs on the assembled SELL form of H (B.hsv, L.hs_*) when
// its pipelined form is memory resident on this grid; *sell (may be null) tells whether it did.
template <class T>
cudaError_t launch_coarse_step(cudaStream_t st, const LevelDev& L, const T* Hc, const T* Sinv,
                               const CoarseStepBufs<T>& B, const CoarseStepParams& P, double* partial, GridSync gs,
                               CoarseStepResult* res, bool* sell = nullptr);


// Failure-detection check: a cooperative launch of min(blocks, co-resident) blocks in which every block but `absent`
// (absent < 0: none) waits at one bounded grid barrier (spin_limit polls); *passed (zeroed by the caller) counts the
// blocks whose wait completed, and *gs.err is set when a wait gave up.
cudaError_t launch_barrier_probe(cudaStream_t st, GridSync gs, double* partial, int blocks, int absent,
                                 unsigned long long spin_limit, int* passed);

}  // namespace nlmg
