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

struct GridSync {
  unsigned* count;   // arrivals at the current barrier (0 at launch); own 128-byte line
  unsigned* gen;     // barrier generation; own 128-byte line
  int* err;          // set when a wait gives up
  double* out;       // 24 reduction results and step lengths published by the last block to arrive
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

template <class T>
cudaError_t launch_hyb_solve(cudaStream_t st, const LevelDev& L, const T* Hc, const T* Sinv, const double* kapc,
                             const double* bs, const double* bp, T* ylam, T* ydiag, T* lam, T* lr, T* lz, T* pa,
                             T* pb, T* lq, T* ldinv, double* dsig, double* dp, double* partial, GridSync gs,
                             double tol, int maxit, PcgResult* res);

}  // namespace nlmg
