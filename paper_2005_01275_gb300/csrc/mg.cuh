// Linear multigrid preconditioner for the level-0 Krylov solves (mg.cu).
//
// Sec. 3.4 preconditions the fine-level Picard and Newton systems with AMG on the Schur complement, which on the
// TPFA fine level is the frozen TPFA matrix A itself. Here one V-cycle on the pressure spaces of the spectral
// hierarchy plays that role: Galerkin operators A_{l+1} = P_l^T A_l P_l (level 1 assembled face by face from the
// fine transmissibilities, in the difference form that keeps the constant mode exact), Chebyshev smoothing
// preconditioned by the (block) diagonal, a dense inverse on the coarsest level; FP32 throughout, inside the FP64
// Krylov iteration. One Krylov solve runs as one CUDA graph whose iterations sit in a device-side conditional
// while node, so no host round trip separates them.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hier.hpp"
#include "kernels.cuh"

namespace nlmg {

constexpr int kMgMaxLevels = 8;
constexpr int kMgMaxCoarse = 128;   // largest coarsest-level system (unknowns, padded): dense inverse in one block
constexpr int kMgDegFine = 2;       // Chebyshev steps before and after the coarse correction, level 0
constexpr int kMgDegCoarse = 2;     // the same on levels 1 .. L-2
constexpr double kMgAlpha = 4.0;    // Chebyshev interval [lam / alpha, lam]
constexpr int kMgMaxDeg = 4;        // Chebyshev steps per smoothing at most (coefficient table size)
constexpr int kTailThreads = 1024;  // threads of the small-level kernel (k_small, one block)
constexpr int kTailMaxCells = 1024; // it starts at the first level l >= 2 with at most this many cells ...
constexpr size_t kTailSmem = 200 * 1024;   // ... whose data from there on fit this much shared memory
constexpr int kTailMaxCopies = 8 * kMgMaxLevels;

// Static structure of the preconditioner (host side, built once per hierarchy).
struct MgHost {
  int L = 0, N = 0;
  int nc[kMgMaxLevels] = {0}, mb[kMgMaxLevels] = {0}, nblk[kMgMaxLevels] = {0};
  std::vector<int> rowptr[kMgMaxLevels], col[kMgMaxLevels], dpos[kMgMaxLevels], mcnt[kMgMaxLevels];
  std::vector<int> asm_off[kMgMaxLevels];
  std::vector<int4> asm_list[kMgMaxLevels];
  std::vector<float> P[kMgMaxLevels];                   // P[l]: transfer l -> l+1, padded
  std::vector<int> agg[kMgMaxLevels], ch_off[kMgMaxLevels], ch[kMgMaxLevels];
};

// Device copy of MgHost (pointers owned by the shared part of a context).
struct MgDev {
  int L = 0, N = 0;
  int nc[kMgMaxLevels] = {0}, mb[kMgMaxLevels] = {0}, nblk[kMgMaxLevels] = {0};
  int *rowptr[kMgMaxLevels] = {nullptr}, *col[kMgMaxLevels] = {nullptr}, *dpos[kMgMaxLevels] = {nullptr},
      *mcnt[kMgMaxLevels] = {nullptr};
  int* asm_off[kMgMaxLevels] = {nullptr};
  int4* asm_list[kMgMaxLevels] = {nullptr};
  float* P[kMgMaxLevels] = {nullptr};
  __nv_bfloat16* Pb[kMgMaxLevels] = {nullptr};          // the same transfers rounded to BF16
  int *agg[kMgMaxLevels] = {nullptr}, *ch_off[kMgMaxLevels] = {nullptr}, *ch[kMgMaxLevels] = {nullptr};
};

// Device scalars of one Krylov solve (one struct per context).
struct MgScal {
  double alpha, beta, omega, rho, rz, rr0, rr, tol2;
  int it, maxit, done, bad;
  unsigned cnt[8];   // arrival counters of the reductions (each reset by its last block)
};

// One contiguous source array of the small-level kernel's copy-in: 16-byte chunks c0 .. to shared byte offset dst.
struct MgTailCopy {
  const void* src;
  unsigned dst, c0;
};

// What the small-level kernel reads, as one device-resident table per context: the level data, its shared-memory
// layout (byte offsets) and copy list (index 0 with FP32 transfers, 1 with BF16).
struct MgTailTab {
  MgDev M;
  float *d[kMgMaxLevels] = {nullptr}, *x[kMgMaxLevels][2] = {{nullptr}};   // global vectors (level t-1 is used)
  int t = 0;
  unsigned o_P[kMgMaxLevels] = {0}, o_choff[kMgMaxLevels] = {0}, o_ch[kMgMaxLevels] = {0}, o_agg[kMgMaxLevels] = {0};
  unsigned o_rowptr[kMgMaxLevels] = {0}, o_col[kMgMaxLevels] = {0}, o_aval[kMgMaxLevels] = {0},
           o_dinv[kMgMaxLevels] = {0}, o_b[kMgMaxLevels] = {0}, o_d[kMgMaxLevels] = {0},
           o_x[kMgMaxLevels][2] = {{0}}, o_cinv = 0, o_coef = 0;
  int ncopies[2] = {0, 0}, nchunks[2] = {0, 0};
  MgTailCopy cp[2][kTailMaxCopies];
};

// Per-context work buffers.
struct MgWork {
  float *a0off = nullptr, *a0diag = nullptr, *a0dinv = nullptr;
  float *aval[kMgMaxLevels] = {nullptr}, *dinv[kMgMaxLevels] = {nullptr};
  float* cinv = nullptr;
  float* lam = nullptr;                                  // [kMgMaxLevels] Gershgorin bounds
  float* coef = nullptr;                                 // [kMgMaxLevels][kMgMaxDeg][2] Chebyshev coefficients
  float *x[kMgMaxLevels][2] = {{nullptr}}, *b[kMgMaxLevels] = {nullptr}, *d[kMgMaxLevels] = {nullptr};
  // Krylov vectors (FP64) and the preconditioned vectors (FP32)
  double *kx = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr, *kb = nullptr;
  double *kv = nullptr, *ks = nullptr, *kt = nullptr, *krh = nullptr, *kpp = nullptr;   // BiCGStab
  float *z[2] = {nullptr, nullptr};
  double* part = nullptr;                                // partial sums of the reductions
  MgScal* sc = nullptr;
  MgScal* h_sc = nullptr;                                // pinned copy
  cudaGraphExec_t g_pcg[2] = {nullptr, nullptr}, g_bicg[2] = {nullptr, nullptr}, g_apply = nullptr;
  MgTailTab* tail = nullptr;   // device copy for the small-level kernel (mg_fill_tail)
  size_t tail_smem = 0;        // its dynamic shared memory
  int bf16 = 0;            // transfers in BF16 (FP32 accumulation) in the setup and V-cycle enqueued next
  int graphs_bf16 = -1;    // the transfer type the captured graphs use (-1: none captured)
  int grid0 = 4096;        // blocks of the level-0 streaming kernels: one full wave, SMs x 8 blocks of 256 threads
  int row_cells = 16384;   // block levels with at least this many cells run the row-parallel kernels
  int graphs_row_cells = -1;   // the row_cells the captured graphs use (-1: none captured)
};

// Builds the preconditioner's structure on the first `levels` levels of H (levels <= H.levels.size()); the coarsest
// of them must have at most kMgMaxCoarse padded unknowns. Returns false and sets err otherwise.
bool mg_build_host(const FineMesh& fm, const Hierarchy& H, int levels, MgHost& M, std::string& err);

// Number of levels of H (from level 0) the preconditioner uses: the smallest prefix whose coarsest level has at most
// kMgMaxCoarse padded unknowns, or 0 if no prefix qualifies.
int mg_levels_for(const Hierarchy& H);

// Enqueues, on stream st, the per-Picard-step setup: FP32 fine values, Galerkin operators, block-diagonal inverses,
// Gershgorin bounds and the coarsest inverse, from the frozen matrix (Tval, diagT) and kappa per cell.
void mg_enqueue_setup(cudaStream_t st, const MgDev& M, const FineDev& F, const MgWork& W, const double* Tval,
                      const double* diagT, const double* kap);

// Enqueues one V-cycle z = B r on stream st for an FP32 right-hand side already in W.b[0] with the first pre-smoothing
// step fused by the caller (x[0][0], d[0] hold it); returns the index i of the level-0 buffer W.x[0][i] that holds z;
// `flag` (may be null) is a device int that makes every kernel return at once when non-zero. With cg_beta the last
// step also forms the flexible CG step length from W.kr, z and z_old = W.z[0] (into W.sc).
int mg_enqueue_vcycle(cudaStream_t st, const MgDev& M, const FineDev& F, const MgWork& W, const int* flag,
                      bool cg_beta);

// Writes W.tail (device memory of sizeof(MgTailTab), allocated by the caller) from M and W, on stream st, and sets
// W.tail_smem. Every array it lists must be allocated in whole 16-byte units.
void mg_fill_tail(cudaStream_t st, const MgDev& M, MgWork& W);

// First level the small-level kernel takes over (levels t .. L-1 and the transfers to and from t-1 in one launch of
// one thread block, out of shared memory), or 0 if the V-cycle runs one kernel per phase throughout.
int mg_tail_level(const MgDev& M);

// Kernels in one V-cycle after its fused first step (for the launch counts of graph replays).
int mg_vcycle_kernels(const MgDev& M);

// The preconditioned Krylov solves as graphs captured once per context (out[0] the start, out[1] a conditional
// while loop over the iterations; tolerance tol2 and cap maxit read from W.sc at run time), and one V-cycle for the
// step calls. Right-hand side W.kb (the solve is for -W.kb), solution W.kx.
cudaError_t mg_capture_pcg(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, const double* Tval,
                           const double* diagT, cudaGraphExec_t* out);
cudaError_t mg_capture_bicgstab(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, const double* jd,
                                const double* Joff, const double* wgt, cudaGraphExec_t* out);
cudaError_t mg_capture_apply(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, cudaGraphExec_t* out);

// Raises the dynamic shared-memory limit of the coarsest-level inversion (once per process).
void mg_set_smem_limits();

}  // namespace nlmg
