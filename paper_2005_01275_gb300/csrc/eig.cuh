// Batched FP64 eigensolver for the setup's local spectral problems (eig.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace nlmg {

constexpr int kMaxEigK = 8;      // eigenpairs per matrix (modes)
constexpr int kMaxEigN = 2048;   // largest matrix

// The ksz[b] smallest eigenpairs of the symmetric nsz[b] x nsz[b] matrices packed row-major in A_all at aoff[b]
// (overwritten). vals[b * (kMaxEigK + 1) + j], j <= ksz[b] (entry ksz[b] is the next eigenvalue, for the gap);
// vecs at voff[b], nsz[b] x ksz[b] row-major. Runs on the current device; returns false and sets err on failure.
bool batched_smallest_eig(int nmat, const std::vector<long long>& aoff, const std::vector<int>& nsz,
                          const std::vector<int>& ksz, std::vector<double>& A_all, std::vector<double>& vals,
                          std::vector<long long>& voff, std::vector<double>& vecs, std::string& err);

}  // namespace nlmg
