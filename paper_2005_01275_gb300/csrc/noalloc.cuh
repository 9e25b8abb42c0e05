// Allocation-free variant of the fine residual (noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "kernels.cuh"

namespace nlmg {

// Largest fine mesh nlmg_fine_residual_noalloc accepts: its per-cell scratch is a fixed device array.
constexpr int kNoallocMaxCells = 1 << 20;

// Resolves (once per device, with that device current) the device address of the file-scope scratch array with
// cudaGetSymbolAddress. The entry point's first call on a device does this, so that first call belongs before any
// stream capture.
bool noalloc_scratch_address(void** out, std::string& err);

// Enqueues kappa + residual + ||R||^2 on stream st using the scratch array; allocates nothing.
bool noalloc_residual(cudaStream_t st, void* scratch, const FineDev& F, const double* p, const double* g,
                      const double* rhs, double* r, double* norm2, int kind, double a, std::string& err);

}  // namespace nlmg
