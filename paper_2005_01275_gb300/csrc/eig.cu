// Batched symmetric eigensolver for the local spectral problems of the setup (eq. local-eigenvalue-problem): the
// k smallest eigenpairs of many small dense FP64 matrices, one thread block per matrix.
//
// Steps per matrix (the same algorithm as the host routine in dense.cpp): Householder reduction to tridiagonal form
// (the trailing block updated in global memory, reflectors kept below the subdiagonal), Sturm-sequence bisection
// for the k+1 smallest eigenvalues, inverse iteration on the tridiagonal matrix with Gram-Schmidt inside clusters,
// then back-transformation by the stored reflectors.
#include <cmath>

#include "eig.cuh"

namespace nlmg {

namespace {

constexpr int kEigThreads = 256;

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

__device__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) cnt++;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) cnt++;
  }
  return cnt;
}

// (T - lam I) x = b by Gaussian elimination with partial pivoting on the tridiagonal (d, e); a0..a2 scratch [n]
__device__ void tri_shift_solve(int n, const double* d, const double* e, double lam, double tiny, double* b,
                                double* a0, double* a1, double* a2) {
  double cd = d[0] - lam, cs = (n > 1) ? e[0] : 0.0, css = 0.0;
  for (int i = 0; i < n - 1; ++i) {
    const double sub = e[i], nd = d[i + 1] - lam, ns = (i + 2 < n) ? e[i + 1] : 0.0;
    if (fabs(sub) > fabs(cd)) {
      const double m = cd / sub;
      a0[i] = sub;
      a1[i] = nd;
      a2[i] = ns;
      const double t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t - m * b[i];
      const double ncd = cs - m * nd, ncs = css - m * ns;
      cd = ncd;
      cs = ncs;
      css = 0.0;
    } else {
      if (cd == 0.0) cd = tiny;
      const double m = sub / cd;
      a0[i] = cd;
      a1[i] = cs;
      a2[i] = css;
      b[i + 1] -= m * b[i];
      cd = nd - m * cs;
      cs = ns - m * css;
      css = 0.0;
    }
  }
  if (cd == 0.0) cd = tiny;
  a0[n - 1] = cd;
  a1[n - 1] = a2[n - 1] = 0.0;
  if (n > 1) a2[n - 2] = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    if (i + 1 < n) s -= a1[i] * b[i + 1];
    if (i + 2 < n) s -= a2[i] * b[i + 2];
    double piv = a0[i];
    if (fabs(piv) < tiny) piv = piv < 0 ? -tiny : tiny;
    b[i] = s / piv;
  }
}

__global__ void __launch_bounds__(kEigThreads) k_batched_eig(int nmat, const long long* __restrict__ aoff,
                                                             const int* __restrict__ nsz, const int* __restrict__ ksz,
                                                             double* A_all, double* work_all,
                                                             const long long* __restrict__ woff,
                                                             double* vals_all, double* vecs_all,
                                                             const long long* __restrict__ voff) {
  extern __shared__ double shm[];
  __shared__ double red[33];
  const int b = blockIdx.x;
  if (b >= nmat) return;
  const int n = nsz[b], k = ksz[b];
  double* A = A_all + aoff[b];
  double* W = work_all + woff[b];     // d[n] e[n] e2[n] beta[n] x[n] a0[n] a1[n] a2[n] Z[n*k]
  double *d = W, *e = W + n, *e2 = W + 2 * n, *beta = W + 3 * n, *x = W + 4 * n, *a0 = W + 5 * n,
         *a1 = W + 6 * n, *a2 = W + 7 * n, *Z = W + 8 * n;
  double* vals = vals_all + (size_t)b * (kMaxEigK + 1);
  double* vecs = vecs_all + voff[b];
  double* v = shm;            // reflector [n]
  double* pw = shm + n;       // p, then w [n]
  const int tid = threadIdx.x, nt = blockDim.x;
  if (n == 1) {
    if (tid == 0) {
      vals[0] = A[0];
      vals[1] = INFINITY;
      vecs[0] = 1.0;
    }
    return;
  }
  // ---- Householder reduction ----
  for (int kk = 0; kk < n - 2; ++kk) {
    const int m = n - kk - 1;
    double part = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double xi = A[(size_t)(kk + 1 + i) * n + kk];
      v[i] = xi;
      part += xi * xi;
    }
    const double nrm2 = block_sum_d(part, red);
    double alpha = sqrt(nrm2);
    if (alpha == 0.0) {
      if (tid == 0) {
        beta[kk] = 0.0;
        e[kk] = 0.0;
      }
      for (int i = tid; i < m; i += nt) A[(size_t)(kk + 1 + i) * n + kk] = 0.0;
      __syncthreads();
      continue;
    }
    const double x0 = v[0];
    if (x0 > 0) alpha = -alpha;
    __syncthreads();
    if (tid == 0) v[0] = x0 - alpha;
    __syncthreads();
    double vp = 0.0;
    for (int i = tid; i < m; i += nt) vp += v[i] * v[i];
    const double vn2 = block_sum_d(vp, red);
    const double bb = 2.0 / vn2;
    // p = bb A22 v : one warp per row, lanes across the row
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int i = warp; i < m; i += nw) {
      const double* Ai = A + (size_t)(kk + 1 + i) * n + kk + 1;
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s += Ai[j] * v[j];
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (lane == 0) pw[i] = bb * s;
    }
    __syncthreads();
    double pvp = 0.0;
    for (int i = tid; i < m; i += nt) pvp += pw[i] * v[i];
    const double pv = block_sum_d(pvp, red);
    for (int i = tid; i < m; i += nt) pw[i] = pw[i] - 0.5 * bb * pv * v[i];
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = idx / m, j = idx - i * m;
      A[(size_t)(kk + 1 + i) * n + kk + 1 + j] -= v[i] * pw[j] + pw[i] * v[j];
    }
    for (int i = tid; i < m; i += nt) A[(size_t)(kk + 1 + i) * n + kk] = v[i];
    if (tid == 0) {
      beta[kk] = bb;
      e[kk] = alpha;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) d[i] = A[(size_t)i * n + i];
  if (tid == 0) {
    e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    beta[n - 2] = 0.0;
    e[n - 1] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i < n - 1; i += nt) e2[i] = e[i] * e[i];
  double tn = 0.0;
  for (int i = tid; i < n; i += nt) {
    double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    tn = fmax(tn, r);
  }
  // block max
  for (int off = 16; off > 0; off >>= 1) tn = fmax(tn, __shfl_down_sync(0xffffffffu, tn, off));
  if ((tid & 31) == 0) red[tid >> 5] = tn;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) t = fmax(t, red[w]);
    red[32] = t;
  }
  __syncthreads();
  const double tnorm = red[32];
  const double eps = 2.220446049250313e-16;
  const double pivmin = fmax(2.2250738585072014e-308, eps * eps * tnorm * tnorm) + 1e-300;
  // ---- bisection: thread j finds eigenvalue j (j <= k) ----
  const int want = min(k + 1, n);
  if (tid < want) {
    double lo = -tnorm, hi = tnorm;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (sturm_count(n, d, e2, mid, pivmin) > tid) hi = mid; else lo = mid;
      if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    }
    vals[tid] = 0.5 * (lo + hi);
  }
  if (tid == 0 && want <= k) vals[k] = INFINITY;
  __syncthreads();
  // ---- inverse iteration (thread 0; vectors in a cluster are orthogonalised against earlier ones) ----
  if (tid == 0) {
    const double tiny = eps * fmax(tnorm, 1e-300);
    const double cluster_tol = 1e-3 * fmax(tnorm, 1e-300);
    int cstart = 0;
    for (int j = 0; j < k; ++j) {
      if (j > 0 && fabs(vals[j] - vals[j - 1]) > cluster_tol) cstart = j;
      unsigned long long s = 0x9E3779B97F4A7C15ull * (unsigned long long)(j + 1);
      for (int i = 0; i < n; ++i) {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        x[i] = ((double)(s >> 11) / 9007199254740992.0) - 0.5;
      }
      for (int it = 0; it < 4; ++it) {
        tri_shift_solve(n, d, e, vals[j], tiny, x, a0, a1, a2);
        for (int q = cstart; q < j; ++q) {
          double dot = 0.0;
          for (int i = 0; i < n; ++i) dot += x[i] * Z[(size_t)i * k + q];
          for (int i = 0; i < n; ++i) x[i] -= dot * Z[(size_t)i * k + q];
        }
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr += x[i] * x[i];
        nr = sqrt(nr);
        if (nr == 0.0) {
          for (int i = 0; i < n; ++i) x[i] = 0.0;
          x[j % n] = 1.0;
          nr = 1.0;
        }
        for (int i = 0; i < n; ++i) x[i] /= nr;
      }
      for (int i = 0; i < n; ++i) Z[(size_t)i * k + j] = x[i];
    }
  }
  __syncthreads();
  // ---- back-transformation y = H_0 ... H_{n-3} z for each vector ----
  for (int j = 0; j < k; ++j) {
    for (int i = tid; i < n; i += nt) x[i] = Z[(size_t)i * k + j];
    __syncthreads();
    for (int kk = n - 3; kk >= 0; --kk) {
      const double bk = beta[kk];
      if (bk == 0.0) continue;
      const int m = n - kk - 1;
      double part = 0.0;
      for (int i = tid; i < m; i += nt) part += A[(size_t)(kk + 1 + i) * n + kk] * x[kk + 1 + i];
      const double dot = bk * block_sum_d(part, red);
      for (int i = tid; i < m; i += nt) x[kk + 1 + i] -= dot * A[(size_t)(kk + 1 + i) * n + kk];
      __syncthreads();
    }
    for (int i = tid; i < n; i += nt) vecs[(size_t)i * k + j] = x[i];
    __syncthreads();
  }
}

}  // namespace

bool batched_smallest_eig(int nmat, const std::vector<long long>& aoff, const std::vector<int>& nsz,
                          const std::vector<int>& ksz, std::vector<double>& A_all, std::vector<double>& vals,
                          std::vector<long long>& voff, std::vector<double>& vecs, std::string& err) {
  if (nmat == 0) return true;
  std::vector<long long> woff(nmat + 1, 0);
  voff.assign(nmat + 1, 0);
  int nmax = 0;
  for (int b = 0; b < nmat; ++b) {
    if (ksz[b] > kMaxEigK || ksz[b] < 1) {
      err = "eigenpair count out of range";
      return false;
    }
    woff[b + 1] = woff[b] + 8LL * nsz[b] + (long long)nsz[b] * ksz[b];
    voff[b + 1] = voff[b] + (long long)nsz[b] * ksz[b];
    nmax = std::max(nmax, nsz[b]);
  }
  if (nmax > kMaxEigN) {
    err = "local eigenproblem larger than the batched solver supports";
    return false;
  }
  double *dA = nullptr, *dW = nullptr, *dV = nullptr, *dvals = nullptr;
  long long *daoff = nullptr, *dwoff = nullptr, *dvoff = nullptr;
  int *dn = nullptr, *dk = nullptr;
  auto fail = [&](cudaError_t e) {
    err = std::string("batched eigensolver: ") + cudaGetErrorString(e);
    for (void* p : {(void*)dA, (void*)dW, (void*)dV, (void*)dvals, (void*)daoff, (void*)dwoff, (void*)dvoff,
                    (void*)dn, (void*)dk})
      if (p) cudaFree(p);
    return false;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&dA, A_all.size() * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dW, woff[nmat] * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dV, std::max<long long>(1, voff[nmat]) * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dvals, (size_t)nmat * (kMaxEigK + 1) * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&daoff, nmat * sizeof(long long))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dwoff, nmat * sizeof(long long))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dvoff, nmat * sizeof(long long))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dn, nmat * sizeof(int))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dk, nmat * sizeof(int))) != cudaSuccess) return fail(e);
  cudaMemcpy(dA, A_all.data(), A_all.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(daoff, aoff.data(), nmat * sizeof(long long), cudaMemcpyHostToDevice);
  cudaMemcpy(dwoff, woff.data(), nmat * sizeof(long long), cudaMemcpyHostToDevice);
  cudaMemcpy(dvoff, voff.data(), nmat * sizeof(long long), cudaMemcpyHostToDevice);
  cudaMemcpy(dn, nsz.data(), nmat * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, ksz.data(), nmat * sizeof(int), cudaMemcpyHostToDevice);
  const size_t shm = 2 * (size_t)nmax * sizeof(double);
  k_batched_eig<<<nmat, kEigThreads, shm>>>(nmat, daoff, dn, dk, dA, dW, dwoff, dvals, dV, dvoff);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  vals.resize((size_t)nmat * (kMaxEigK + 1));
  vecs.resize(voff[nmat]);
  cudaMemcpy(vals.data(), dvals, vals.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (!vecs.empty()) cudaMemcpy(vecs.data(), dV, vecs.size() * sizeof(double), cudaMemcpyDeviceToHost);
  for (void* p : {(void*)dA, (void*)dW, (void*)dV, (void*)dvals, (void*)daoff, (void*)dwoff, (void*)dvoff,
                  (void*)dn, (void*)dk})
    cudaFree(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  return true;
}

}  // namespace nlmg
