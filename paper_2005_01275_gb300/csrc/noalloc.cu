// nlmg_fine_residual_noalloc: the fine TPFA residual and its squared norm for callers that must not allocate
// device memory at call time (no cudaMalloc, cudaFree or allocating library routine is called here).
//
// The kernels are the ones of nlmg_fine_residual (k_kappa, then k_residual with its deterministic last-block
// reduction); what differs is where their scratch lives: kappa per cell and the per-block partial sums sit in one
// file-scope device array of fixed size instead of buffers the context allocated.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/nlmg.h"
#include "kernels.cuh"
#include "noalloc.cuh"

namespace nlmg {

namespace {

struct NoallocScratch {
  double kap[kNoallocMaxCells];     // kappa(p) per cell
  double partial[kMaxBlocks * 4];   // per-block partial sums of the reduction
  unsigned counter;                 // arrivals of the last-block reduction (must be 0 when a launch starts)
};

// Lives on every device that loads this library until the process exits (about 8.1 MiB).
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch* g_addr[kMaxDevices] = {nullptr};

}  // namespace

// Device address of the scratch array on the current device, resolved once per device. Nothing in the array needs
// clearing here: kappa and the partial sums are written before they are read, and the arrival counter is zeroed on
// the caller's stream before every launch (and left at zero by the reduction's last block).
bool noalloc_scratch_address(void** out, std::string& err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return false;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return false;
    }
    g_addr[dev] = (NoallocScratch*)p;
  }
  *out = g_addr[dev];
  return true;
}

bool noalloc_residual(cudaStream_t st, void* scratch, const FineDev& F, const double* p, const double* g,
                      const double* rhs, double* r, double* norm2, int kind, double a, std::string& err) {
  NoallocScratch* S = (NoallocScratch*)scratch;
  cudaError_t e = cudaMemsetAsync(&S->counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) {
    err = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
    return false;
  }
  launch_kappa(st, F.N, p, nullptr, 0.0, const_cast<double*>(p), S->kap, nullptr, kind, a);
  Reduce red{S->partial, &S->counter, norm2};
  launch_residual(st, F, p, S->kap, nullptr, g, rhs, r, nullptr, nullptr, nullptr, nullptr, red);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

}  // namespace nlmg
