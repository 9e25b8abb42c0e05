// Linear multigrid preconditioner for the level-0 Krylov solves (see mg.cuh), and the preconditioned CG / BiCGStab
// that use it, each captured once per context as CUDA graphs with a device-side conditional while loop.
//
// Every reduction is deterministic: per-block partial sums in a fixed tree, then the grid's last block adds the
// partials in block order (the arrival counter is reset by that block, so graphs replay). Maxima are exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "mg.cuh"

namespace nlmg {

namespace {

static_assert(kMgDegFine <= kMgMaxDeg && kMgDegCoarse <= kMgMaxDeg, "Chebyshev coefficient table too small");
static_assert(kMgMaxLevels * kMgMaxDeg <= 32, "the coefficient table kernel runs one warp");

constexpr int kT = 256;               // threads per block of the preconditioner kernels
constexpr int kMaxRedBlocks = 1024;   // grid cap of the reduction kernels (partials summed by one block)

#define MG_MB_SWITCH(mb, CALL)                                                     \
  switch (mb) {                                                                    \
    case 1: { constexpr int MB = 1; CALL; } break;                                 \
    case 2: { constexpr int MB = 2; CALL; } break;                                 \
    case 3: { constexpr int MB = 3; CALL; } break;                                 \
    case 4: { constexpr int MB = 4; CALL; } break;                                 \
    case 5: { constexpr int MB = 5; CALL; } break;                                 \
    case 6: { constexpr int MB = 6; CALL; } break;                                 \
    case 7: { constexpr int MB = 7; CALL; } break;                                 \
    default: { constexpr int MB = 8; CALL; } break;                                \
  }

inline int blocks_for(long n, int cap = 1 << 20) {
  long b = (n + kT - 1) / kT;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// ---------------------------------------------------------------------------------------------------------------
// reductions

// Sums NV values over the grid: block tree sums to part[block][k]; the last block to arrive adds the partials in block
// order (thread t takes partials t, t + blockDim, ...; then a fixed tree) and returns true in every one of its
// threads with the sums in out (shared). The counter is left at zero.
template <int NV>
__device__ bool reduce_last(double (&v)[NV], double* part, unsigned* cnt, double* out) {
  __shared__ double sh[NV][kT / 32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) sh[k][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < kT / 32; ++w) a += sh[k][w];
      part[(size_t)blockIdx.x * NV + k] = a;
    }
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kT) a += __ldcg(&part[(size_t)b * NV + k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) sh[k][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < kT / 32; ++w) a += sh[k][w];
      out[k] = a;
    }
    *cnt = 0u;
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ void atomic_max_pos(float* addr, float v) {
  // non-negative floats order like their bit patterns
  atomicMax((unsigned*)addr, __float_as_uint(v));
}

// Chebyshev coefficients of step k on [lam / alpha, lam] (see oracle/precond.py): k = 0 -> (0, 1 / theta);
// k >= 1 -> (rho_k rho_{k-1}, 2 rho_k / delta).
__device__ __forceinline__ void cheb_coef(float lam, int k, float& c1, float& c2) {
  const double lmax = lam, lmin = lam / kMgAlpha;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  if (k == 0) {
    c1 = 0.0f;
    c2 = (float)(1.0 / theta);
    return;
  }
  double rho = 1.0 / sigma, rho_prev = rho;
  for (int i = 1; i <= k; ++i) {
    rho_prev = rho;
    rho = 1.0 / (2.0 * sigma - rho);
  }
  c1 = (float)(rho * rho_prev);
  c2 = (float)(2.0 * rho / delta);
}

// The coefficients of every level and step, computed once per setup from the Gershgorin bounds (k_cheb_table):
// tab[(l * kMgMaxDeg + k) * 2 + {0, 1}] = (c1, c2) of cheb_coef.
__device__ __forceinline__ void cheb_tab(const float* __restrict__ tab, int l, int k, float& c1, float& c2) {
  c1 = tab[(l * kMgMaxDeg + k) * 2];
  c2 = tab[(l * kMgMaxDeg + k) * 2 + 1];
}

__device__ __forceinline__ bool stop(const int* done) { return done && *((volatile const int*)done) != 0; }

// Programmatic dependent launch: wait until the preceding kernel of the stream (or graph edge) has finished and its
// writes are visible, then let the next kernel start its launch (it waits the same way before it reads anything).
// Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float pval(const float* __restrict__ p, size_t i) { return p[i]; }
__device__ __forceinline__ float pval(const __nv_bfloat16* __restrict__ p, size_t i) { return __bfloat162float(p[i]); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ---------------------------------------------------------------------------------------------------------------
// setup kernels (once per frozen matrix)

// FP32 copy of the level-0 matrix (off-diagonal entries -T in the SELL layout, diagonal, its inverse) and the
// Gershgorin bound max_K (A_KK + sum_L T_KL) / A_KK of D^-1 A.
__global__ void k_fine_vals(FineDev F, const double* __restrict__ Tval, const double* __restrict__ diagT,
                            float* __restrict__ a0off, float* __restrict__ a0diag, float* __restrict__ a0dinv,
                            float* lam) {
  pdl_start();
  float g = 0.0f;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    const int w = F.sell_w[K >> 5];
    int e = F.sell_off[K >> 5] + (K & 31);
    double s = 0.0;
    for (int j = 0; j < w; ++j, e += 32) {
      const double t = Tval[e];
      a0off[e] = (float)(-t);
      s += t;
    }
    const double dg = diagT[K];
    a0diag[K] = (float)dg;
    a0dinv[K] = (float)(1.0 / dg);
    g = fmaxf(g, (float)((dg + s) / dg));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) g = fmaxf(g, __shfl_down_sync(0xffffffffu, g, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(&lam[0], g);
}

// Level-1 Galerkin blocks from the fine faces, one warp per block: lane t takes contributions t, t + 32, ... of the
// block's list and accumulates the whole MB x MB block; a fixed shuffle tree then adds the lanes' blocks. The
// contributions (K, L, e, type): 0 interior face inside the aggregate, T (P_K - P_L)(P_K - P_L)^T; 1 face to another
// aggregate seen from this one's cell K, T P_K P_K^T; 2 the off-diagonal part, -T P_K P_L^T; 3 Dirichlet face (L = its
// entry in the Dirichlet list), h P_K P_K^T with h = kappa_K Ups_K.
template <int MB, class PT>
__global__ void k_asm1(int nblk, const int* __restrict__ off, const int4* __restrict__ list,
                       const PT* __restrict__ P0, const double* __restrict__ Tval, const double* __restrict__ kap,
                       const double* __restrict__ dir_ups, float* __restrict__ aval) {
  pdl_start();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = warp; b < nblk; b += nw) {
    float acc[MB * MB];
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) acc[i] = 0.0f;
    for (int c = off[b] + lane; c < off[b + 1]; c += 32) {
      const int4 t = list[c];
      float pk[MB], pl[MB];
#pragma unroll
      for (int j = 0; j < MB; ++j) pk[j] = pval(P0, (size_t)t.x * MB + j);
      float w;
      if (t.w == 3) {
        w = (float)(kap[t.x] * dir_ups[t.y]);
#pragma unroll
        for (int j = 0; j < MB; ++j) pl[j] = pk[j];
      } else {
        w = (float)Tval[t.z];
#pragma unroll
        for (int j = 0; j < MB; ++j) pl[j] = pval(P0, (size_t)t.y * MB + j);
        if (t.w == 0) {
#pragma unroll
          for (int j = 0; j < MB; ++j) {
            pk[j] -= pl[j];
            pl[j] = pk[j];
          }
        } else if (t.w == 1) {
#pragma unroll
          for (int j = 0; j < MB; ++j) pl[j] = pk[j];
        } else {
          w = -w;
        }
      }
#pragma unroll
      for (int u = 0; u < MB; ++u)
#pragma unroll
        for (int v = 0; v < MB; ++v) acc[u * MB + v] = fmaf(w * pk[u], pl[v], acc[u * MB + v]);
    }
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) acc[i] = warp_sum(acc[i]);
#pragma unroll
    for (int i = 0; i < MB * MB; ++i)
      if ((i & 31) == lane) aval[(size_t)b * MB * MB + i] = acc[i];
  }
}

// Unit diagonal on the padded modes of every diagonal block of level l (cells with fewer modes than mb).
__global__ void k_pad_diag(int nc, int mb, const int* __restrict__ dpos, const int* __restrict__ mcnt,
                           float* __restrict__ aval) {
  pdl_start();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    float* B = aval + (size_t)dpos[c] * mb * mb;
    for (int u = mcnt[c]; u < mb; ++u) {
      for (int v = 0; v < mb; ++v) B[u * mb + v] = B[v * mb + u] = 0.0f;
      B[u * mb + u] = 1.0f;
    }
  }
}

// Level-l Galerkin blocks (l >= 2) from the level-(l-1) blocks: block (A, B) = sum over (c, d) with agg(c) = A,
// agg(d) = B of P_c^T A_cd P_d, P_c the mbf x MB transfer block of level-(l-1) cell c. One warp per block, lanes
// taking the contributions in turn, then a fixed shuffle tree.
template <int MB, class PT>
__global__ void k_asml(int nblk, int mbf, const int* __restrict__ off, const int4* __restrict__ list,
                       const PT* __restrict__ Pf, const float* __restrict__ afine, float* __restrict__ aval) {
  pdl_start();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = warp; b < nblk; b += nw) {
    float acc[MB * MB];
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) acc[i] = 0.0f;
    for (int c = off[b] + lane; c < off[b + 1]; c += 32) {
      const int4 t = list[c];   // (source block, c, d, -)
      const float* As = afine + (size_t)t.x * mbf * mbf;
      const size_t pc = (size_t)t.y * mbf * MB, pd = (size_t)t.z * mbf * MB;
      for (int i = 0; i < mbf; ++i) {
        float ti[MB];
#pragma unroll
        for (int v = 0; v < MB; ++v) ti[v] = 0.0f;
        for (int j = 0; j < mbf; ++j) {
          const float a = As[i * mbf + j];
#pragma unroll
          for (int v = 0; v < MB; ++v) ti[v] = fmaf(a, pval(Pf, pd + j * MB + v), ti[v]);
        }
#pragma unroll
        for (int u = 0; u < MB; ++u) {
          const float pu = pval(Pf, pc + i * MB + u);
#pragma unroll
          for (int v = 0; v < MB; ++v) acc[u * MB + v] = fmaf(pu, ti[v], acc[u * MB + v]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) acc[i] = warp_sum(acc[i]);
#pragma unroll
    for (int i = 0; i < MB * MB; ++i)
      if ((i & 31) == lane) aval[(size_t)b * MB * MB + i] = acc[i];
  }
}

// Inverse of each diagonal block of a block level (Gauss-Jordan in FP64 registers, no pivoting: the blocks are
// symmetric positive definite) and the Gershgorin bound max over rows of sum |D^-1 A| (one thread per cell).
template <int MB>
__global__ void k_block_inv(int nc, const int* __restrict__ rowptr, const int* __restrict__ dpos,
                            const float* __restrict__ aval, float* __restrict__ dinv, float* lam) {
  pdl_start();
  float g = 0.0f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    double A[MB * MB];
    const float* B = aval + (size_t)dpos[c] * MB * MB;
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) A[i] = B[i];
#pragma unroll
    for (int k = 0; k < MB; ++k) {
      const double dk = 1.0 / A[k * MB + k];
      A[k * MB + k] = 1.0;
#pragma unroll
      for (int j = 0; j < MB; ++j) A[k * MB + j] *= dk;
#pragma unroll
      for (int i = 0; i < MB; ++i) {
        if (i == k) continue;
        const double f = A[i * MB + k];
        A[i * MB + k] = 0.0;
#pragma unroll
        for (int j = 0; j < MB; ++j) A[i * MB + j] -= f * A[k * MB + j];
      }
    }
    float Di[MB * MB];
#pragma unroll
    for (int i = 0; i < MB * MB; ++i) {
      Di[i] = (float)A[i];
      dinv[(size_t)c * MB * MB + i] = Di[i];
    }
    float rs[MB];
#pragma unroll
    for (int u = 0; u < MB; ++u) rs[u] = 0.0f;
    for (int q = rowptr[c]; q < rowptr[c + 1]; ++q) {
      const float* Bq = aval + (size_t)q * MB * MB;
      float Bl[MB * MB];
#pragma unroll
      for (int i = 0; i < MB * MB; ++i) Bl[i] = Bq[i];
#pragma unroll
      for (int u = 0; u < MB; ++u)
#pragma unroll
        for (int v = 0; v < MB; ++v) {
          float t = 0.0f;
#pragma unroll
          for (int w = 0; w < MB; ++w) t = fmaf(Di[u * MB + w], Bl[w * MB + v], t);
          rs[u] += fabsf(t);
        }
    }
#pragma unroll
    for (int u = 0; u < MB; ++u) g = fmaxf(g, rs[u]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) g = fmaxf(g, __shfl_down_sync(0xffffffffu, g, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(lam, g);
}

// Chebyshev coefficient table of every level and step from the Gershgorin bounds (one thread per entry).
__global__ void k_cheb_table(const float* __restrict__ lam, float* __restrict__ tab) {
  pdl_start();
  const int t = threadIdx.x;
  if (t >= kMgMaxLevels * kMgMaxDeg) return;
  const int l = t / kMgMaxDeg, k = t % kMgMaxDeg;
  float c1 = 0.0f, c2 = 0.0f;
  if (lam[l] > 0.0f) cheb_coef(lam[l], k, c1, c2);
  tab[2 * t] = c1;
  tab[2 * t + 1] = c2;
}

// Dense inverse of the coarsest level (n = nc * mb <= kMgMaxCoarse) in one block: the blocks assembled into an
// n x n FP64 matrix in shared memory, in-place Gauss-Jordan (symmetric positive definite, no pivoting).
__global__ void k_coarse_inv(int nc, int mb, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const float* __restrict__ aval, float* __restrict__ cinv) {
  pdl_start();
  extern __shared__ double S[];   // n * n + n
  const int n = nc * mb;
  double* colk = S + n * n;
  __shared__ double piv;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) S[i] = 0.0;
  __syncthreads();
  for (int c = 0; c < nc; ++c)
    for (int q = rowptr[c]; q < rowptr[c + 1]; ++q) {
      const int d = col[q];
      for (int idx = threadIdx.x; idx < mb * mb; idx += blockDim.x) {
        const int u = idx / mb, v = idx % mb;
        S[(c * mb + u) * n + d * mb + v] = aval[(size_t)q * mb * mb + idx];
      }
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      piv = 1.0 / S[k * n + k];
      S[k * n + k] = 1.0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) S[k * n + j] *= piv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = i == k ? 0.0 : S[i * n + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      if (i == k) continue;
      if (j == k)
        S[idx] = -colk[i] * S[k * n + k];
      else
        S[idx] -= colk[i] * S[k * n + j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) cinv[i] = (float)S[i];
}

// ---------------------------------------------------------------------------------------------------------------
// V-cycle kernels

// One Chebyshev step on level 0: res = b - A x_in, d = c1 d + c2 D^-1 res, x_out = x_in + d (x_in is gathered by the
// neighbours, so the new iterate goes to the other buffer).
__device__ __forceinline__ float cheb0_cell(const FineDev& F, const float* __restrict__ a0off,
                                            const float* __restrict__ a0diag, const float* __restrict__ a0dinv,
                                            const float* __restrict__ b, const float* __restrict__ xin,
                                            float* __restrict__ xout, float* __restrict__ d, float c1, float c2, int k,
                                            int K) {
  const int w = F.sell_w[K >> 5];
  int e = F.sell_off[K >> 5] + (K & 31);
  const float xk = xin[K];
  float ax = a0diag[K] * xk;
  for (int j = 0; j < w; ++j, e += 32) ax = fmaf(a0off[e], xin[F.nbr[e]], ax);
  const float res = b[K] - ax;
  const float dn = (k == 0 ? 0.0f : c1 * d[K]) + c2 * a0dinv[K] * res;
  d[K] = dn;
  const float xn = xk + dn;
  xout[K] = xn;
  return xn;
}

__global__ void k_cheb0(FineDev F, const float* __restrict__ a0off, const float* __restrict__ a0diag,
                        const float* __restrict__ a0dinv, const float* __restrict__ b, const float* __restrict__ xin,
                        float* __restrict__ xout, float* __restrict__ d, const float* __restrict__ lam, int k,
                        const int* done) {
  pdl_start();
  if (stop(done)) return;
  float c1, c2;
  cheb_tab(lam, 0, k, c1, c2);
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x)
    (void)cheb0_cell(F, a0off, a0diag, a0dinv, b, xin, xout, d, c1, c2, k, K);
}

// The last Chebyshev step of level 0 (z = xout) fused with the flexible CG step length: rz_new = (r, z),
// beta = (r, z - z_old) / rz (0 on the first step), which equals the plain rz_new / rz for a fixed linear
// preconditioner and tolerates the FP32 rounding of the V-cycle. At most kMaxRedBlocks blocks.
__global__ void k_cheb0_beta(FineDev F, const float* __restrict__ a0off, const float* __restrict__ a0diag,
                             const float* __restrict__ a0dinv, const float* __restrict__ b,
                             const float* __restrict__ xin, float* __restrict__ xout, float* __restrict__ d,
                             const float* __restrict__ lam, int k, const double* __restrict__ r,
                             const float* __restrict__ zold, double* part, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done)) return;
  float c1, c2;
  cheb_tab(lam, 0, k, c1, c2);
  const bool first = sc->it == 0;
  double v[2] = {0.0, 0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    const float z = cheb0_cell(F, a0off, a0diag, a0dinv, b, xin, xout, d, c1, c2, k, K);
    v[0] = fma(r[K], (double)z, v[0]);
    if (!first) v[1] = fma(r[K], (double)zold[K], v[1]);
  }
  __shared__ double out[2];
  if (reduce_last<2>(v, part, &sc->cnt[1], out) && threadIdx.x == 0) {
    sc->beta = first ? 0.0 : (out[0] - out[1]) / sc->rz;
    sc->rz = out[0];
  }
}

// Loads of the vectors a V-cycle writes: ordinary loads, or (CG) through L2 with ld.global.cg for data another CTA
// wrote in the same launch.
template <bool CG>
__device__ __forceinline__ float ldv(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// (A x)_u of block-level cell c, one warp per cell: lane = slot * 8 + u, the four slots take every fourth block of
// the row; a shuffle tree adds the slots, so every lane with component u < MB holds (A x)_u. The blocks are taken in
// batches of RB per slot whose column indices, then matrix and vector entries, are all loaded before the first
// product: on the small levels few warps are in flight, and a row costs two dependent memory round trips per batch
// instead of two per block. The products are added in block order either way.
template <int MB, bool CG>
__device__ __forceinline__ float row_ax(int c, int lane, const int* __restrict__ rowptr, const int* __restrict__ col,
                                        const float* __restrict__ aval, const float* x) {
  constexpr int RB = MB >= 8 ? 2 : (MB >= 4 ? 4 : 8);
  const int slot = lane >> 3, u = lane & 7;
  float ax = 0.0f;
  if (u < MB) {
    const int q1 = rowptr[c + 1];
    for (int qb = rowptr[c] + slot; qb < q1; qb += 4 * RB) {
      int cq[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) cq[j] = qb + 4 * j < q1 ? col[qb + 4 * j] : -1;
      float bv[RB][MB], xv[RB][MB];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const float* Bq = aval + (size_t)(qb + 4 * j) * MB * MB + u * MB;
        const float* xd = x + (size_t)(cq[j] < 0 ? 0 : cq[j]) * MB;
#pragma unroll
        for (int v = 0; v < MB; ++v) {
          bv[j][v] = cq[j] >= 0 ? Bq[v] : 0.0f;
          xv[j][v] = cq[j] >= 0 ? ldv<CG>(xd + v) : 0.0f;
        }
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (cq[j] >= 0) {
#pragma unroll
          for (int v = 0; v < MB; ++v) ax = fmaf(bv[j][v], xv[j][v], ax);
        }
    }
  }
  ax += __shfl_xor_sync(0xffffffffu, ax, 8);
  ax += __shfl_xor_sync(0xffffffffu, ax, 16);
  return ax;
}

// One Chebyshev step on block level l (coefficients c1, c2 of step k): res = b - A x_in, d = c1 d + c2 D^-1 res,
// x_out = x_in + d; warps w0, w0 + nw, ... take one cell each (see row_ax).
template <int MB, bool CG>
__device__ __forceinline__ void chebl_body(int w0, int nw, int nc, const int* __restrict__ rowptr,
                                           const int* __restrict__ col, const float* __restrict__ aval,
                                           const float* __restrict__ dinv, const float* b, const float* xin,
                                           float* xout, float* d, float c1, float c2, int k) {
  const int lane = threadIdx.x & 31, u = lane & 7;
  for (int c = w0; c < nc; c += nw) {
    const float ax = row_ax<MB, CG>(c, lane, rowptr, col, aval, xin);
    const float res = u < MB ? ldv<CG>(b + (size_t)c * MB + u) - ax : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int v = 0; v < MB; ++v) {
      const float rv = __shfl_sync(0xffffffffu, res, v);
      if (u < MB) s = fmaf(dinv[(size_t)c * MB * MB + u * MB + v], rv, s);
    }
    if (lane < MB) {
      const size_t i = (size_t)c * MB + u;
      const float dn = (k == 0 ? 0.0f : c1 * ldv<CG>(d + i)) + c2 * s;
      d[i] = dn;
      xout[i] = ldv<CG>(xin + i) + dn;
    }
  }
}

// Residual b - A x of a block level, one warp per cell.
template <int MB, bool CG>
__device__ __forceinline__ void resl_body(int w0, int nw, int nc, const int* __restrict__ rowptr,
                                          const int* __restrict__ col, const float* __restrict__ aval, const float* b,
                                          const float* x, float* res) {
  const int lane = threadIdx.x & 31;
  for (int c = w0; c < nc; c += nw) {
    const float ax = row_ax<MB, CG>(c, lane, rowptr, col, aval, x);
    if (lane < MB) res[(size_t)c * MB + lane] = ldv<CG>(b + (size_t)c * MB + lane) - ax;
  }
}

// Restriction of a residual (mbf per cell on level l) to level l+1 (mb per cell), one warp per level-(l+1) cell A:
// lane = k * 8 + u takes component u of children k, k + 4, ...; a shuffle tree adds the lanes. `first` adds the first
// Chebyshev step of level l+1 (x = c2 D^-1 b, d = x).
template <class PT, bool CG>
__device__ __forceinline__ void restr_body(int w0, int nw, int mbf, const float* res, const PT* __restrict__ Pl,
                                           const int* __restrict__ ch_off, const int* __restrict__ ch, int ncc,
                                           int mb, float* bc, const float* __restrict__ dinvc, float* xc, float* dc,
                                           float c2, int first) {
  const int lane = threadIdx.x & 31, grp = lane >> 3, u = lane & 7;
  // one value per child (level 0): lanes take children one each; else eight lanes per child
  const int cstep = mbf == 1 ? 32 : 4, c0 = mbf == 1 ? lane : grp, uu = mbf == 1 ? 0 : u;
  for (int A = w0; A < ncc; A += nw) {
    float acc[kMaxM];
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) acc[j] = 0.0f;
    if (uu < mbf) {
      // children in pairs, both loaded before the products (see row_ax); products in child order
      const int t1 = ch_off[A + 1];
      for (int t = ch_off[A] + c0; t < t1; t += 2 * cstep) {
        const bool two = t + cstep < t1;
        const int ca = ch[t], cb = two ? ch[t + cstep] : ca;
        const float ra = ldv<CG>(res + (size_t)ca * mbf + uu), rb = ldv<CG>(res + (size_t)cb * mbf + uu);
        const size_t pa = ((size_t)ca * mbf + uu) * mb, pb = ((size_t)cb * mbf + uu) * mb;
        float Pa[kMaxM], Pb[kMaxM];
#pragma unroll
        for (int j = 0; j < kMaxM; ++j)
          if (j < mb) {
            Pa[j] = pval(Pl, pa + j);
            Pb[j] = pval(Pl, pb + j);
          }
#pragma unroll
        for (int j = 0; j < kMaxM; ++j)
          if (j < mb) acc[j] = fmaf(Pa[j], ra, acc[j]);
        if (two) {
#pragma unroll
          for (int j = 0; j < kMaxM; ++j)
            if (j < mb) acc[j] = fmaf(Pb[j], rb, acc[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxM; ++j)
      if (j < mb) acc[j] = warp_sum(acc[j]);
    if (lane < mb) {
      float bj = 0.0f;
#pragma unroll
      for (int j = 0; j < kMaxM; ++j)
        if (j == lane) bj = acc[j];
      bc[(size_t)A * mb + lane] = bj;
      if (first) {
        const float* Dc = dinvc + (size_t)A * mb * mb + lane * mb;
        float s = 0.0f;
#pragma unroll
        for (int v = 0; v < kMaxM; ++v)
          if (v < mb) s = fmaf(Dc[v], acc[v], s);
        const float dn = c2 * s;
        dc[(size_t)A * mb + lane] = dn;
        xc[(size_t)A * mb + lane] = dn;
      }
    }
  }
}

// x += P e on a block level (one thread per cell and component; threads i0, i0 + ni, ...).
template <class PT, bool CG>
__device__ __forceinline__ void prol_body(long i0, long ni, int nc, int mbf, int mb, const PT* __restrict__ Pl,
                                          const int* __restrict__ agg, const float* e, float* x) {
  const long total = (long)nc * mbf;
  for (long i = i0; i < total; i += ni) {
    const int c = (int)(i / mbf);
    const float* ea = e + (size_t)agg[c] * mb;
    float s = ldv<CG>(x + i);
    for (int j = 0; j < mb; ++j) s = fmaf(pval(Pl, (size_t)i * mb + j), ldv<CG>(ea + j), s);
    x[i] = s;
  }
}

// Coarsest level: x = C^-1 b with the dense inverse (threads i0, i0 + ni, ... take one row each).
template <bool CG>
__device__ __forceinline__ void coarse_solve_body(int i0, int ni, int n, const float* __restrict__ cinv,
                                                  const float* b, float* x) {
  for (int i = i0; i < n; i += ni) {
    float s = 0.0f;
    for (int j = 0; j < n; ++j) s = fmaf(cinv[(size_t)i * n + j], ldv<CG>(b + j), s);
    x[i] = s;
  }
}

__device__ __forceinline__ int gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int nwarps() { return (gridDim.x * blockDim.x) >> 5; }

template <int MB>
__global__ void k_chebl(int nc, const int* __restrict__ rowptr, const int* __restrict__ col,
                        const float* __restrict__ aval, const float* __restrict__ dinv, const float* __restrict__ b,
                        const float* __restrict__ xin, float* __restrict__ xout, float* __restrict__ d,
                        const float* __restrict__ lam, int l, int k, const int* done) {
  pdl_start();
  if (stop(done)) return;
  float c1, c2;
  cheb_tab(lam, l, k, c1, c2);
  chebl_body<MB, false>(gwarp(), nwarps(), nc, rowptr, col, aval, dinv, b, xin, xout, d, c1, c2, k);
}

template <int MB>
__global__ void k_resl(int nc, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const float* __restrict__ aval, const float* __restrict__ b, const float* __restrict__ x,
                       float* __restrict__ res, const int* done) {
  pdl_start();
  if (stop(done)) return;
  resl_body<MB, false>(gwarp(), nwarps(), nc, rowptr, col, aval, b, x, res);
}

template <class PT>
__global__ void k_restr(int mbf, const float* __restrict__ res, const PT* __restrict__ Pl,
                        const int* __restrict__ ch_off, const int* __restrict__ ch, int ncc, int mb,
                        float* __restrict__ bc, const float* __restrict__ dinvc, float* __restrict__ xc,
                        float* __restrict__ dc, const float* __restrict__ lam, int lc, int first, const int* done) {
  pdl_start();
  if (stop(done)) return;
  float c1 = 0.0f, c2 = 0.0f;
  if (first) cheb_tab(lam, lc, 0, c1, c2);
  restr_body<PT, false>(gwarp(), nwarps(), mbf, res, Pl, ch_off, ch, ncc, mb, bc, dinvc, xc, dc, c2, first);
}

// Level-0 residual b - A x (FP32), one thread per cell.
__global__ void k_res0(FineDev F, const float* __restrict__ a0off, const float* __restrict__ a0diag,
                       const float* __restrict__ b, const float* __restrict__ x, float* __restrict__ res,
                       const int* done) {
  pdl_start();
  if (stop(done)) return;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    const int w = F.sell_w[K >> 5];
    int e = F.sell_off[K >> 5] + (K & 31);
    float ax = a0diag[K] * x[K];
    for (int j = 0; j < w; ++j, e += 32) ax = fmaf(a0off[e], x[F.nbr[e]], ax);
    res[K] = b[K] - ax;
  }
}

__global__ void k_coarse_solve(int n, const float* __restrict__ cinv, const float* __restrict__ b,
                               float* __restrict__ x, const int* done) {
  pdl_start();
  if (stop(done)) return;
  coarse_solve_body<false>(threadIdx.x, blockDim.x, n, cinv, b, x);
}

// x_0 += P e on level 0 (per fine cell) and on a block level (per cell and component).
template <class PT>
__global__ void k_pro0(int N, int mb, const PT* __restrict__ P0, const int* __restrict__ agg,
                       const float* __restrict__ e, float* __restrict__ x, const int* done) {
  pdl_start();
  if (stop(done)) return;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    const float* ea = e + (size_t)agg[K] * mb;
    float s = x[K];
    for (int j = 0; j < mb; ++j) s = fmaf(pval(P0, (size_t)K * mb + j), ea[j], s);
    x[K] = s;
  }
}
template <class PT>
__global__ void k_prol(int nc, int mbf, int mb, const PT* __restrict__ Pl, const int* __restrict__ agg,
                       const float* __restrict__ e, float* __restrict__ x, const int* done) {
  pdl_start();
  if (stop(done)) return;
  prol_body<PT, false>((long)blockIdx.x * blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x, nc, mbf, mb, Pl,
                       agg, e, x);
}

// MB consecutive floats from p into v: 16-byte loads when MB % 4 == 0, 8-byte loads when MB is even (the caller
// guarantees p is aligned accordingly: every array here is its own allocation, and a block row or a cell's vector
// segment starts at a multiple of MB floats).
template <int MB>
__device__ __forceinline__ void ld_seg(const float* p, float (&v)[MB]) {
  if constexpr (MB % 4 == 0) {
#pragma unroll
    for (int k = 0; k < MB / 4; ++k) {
      const float4 t = reinterpret_cast<const float4*>(p)[k];
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  } else if constexpr (MB % 2 == 0) {
#pragma unroll
    for (int k = 0; k < MB / 2; ++k) {
      const float2 t = reinterpret_cast<const float2*>(p)[k];
      v[2 * k] = t.x;
      v[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < MB; ++k) v[k] = p[k];
  }
}

// MB consecutive BF16 transfer entries from p, widened to float: 4-byte pair loads when MB is even.
template <int MB>
__device__ __forceinline__ void ld_seg(const __nv_bfloat16* p, float (&v)[MB]) {
  if constexpr (MB % 2 == 0) {
#pragma unroll
    for (int k = 0; k < MB / 2; ++k) {
      const float2 t = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[k]);
      v[2 * k] = t.x;
      v[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < MB; ++k) v[k] = __bfloat162float(p[k]);
  }
}

// Row-parallel forms of the block-level smoothing step and residual (the per-level kernels of the V-cycle; the
// shared-memory tail keeps the warp-per-cell bodies above): one thread per cell component, cell c = 32 g + t / MB and
// component u = t % MB for thread t of a block of 32 MB threads, so a block holds whole cells; blocks take groups g
// gridDim.x apart. A thread reads row u of each block of the cell's row in block order and the block column's x
// segment, with vector loads, the column indices of kRowBatch blocks before their entries. The warp-per-cell form
// leaves 8 - MB of every 8 lanes idle and runs one cell per warp; here every lane is busy and a warp covers 32 / MB
// cells.
template <int MB>
__device__ __forceinline__ float row_ax_u(int c, int u, const int* __restrict__ rowptr, const int* __restrict__ col,
                                          const float* __restrict__ aval, const float* __restrict__ x) {
  constexpr int RB = MB <= 4 ? 8 : 4;
  float ax = 0.0f;
  const int q1 = rowptr[c + 1];
  for (int qb = rowptr[c]; qb < q1; qb += RB) {
    int cq[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) cq[j] = qb + j < q1 ? col[qb + j] : -1;
    float a[RB][MB], xv[RB][MB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      if (cq[j] >= 0) {
        ld_seg<MB>(aval + ((size_t)(qb + j) * MB + u) * MB, a[j]);
        ld_seg<MB>(x + (size_t)cq[j] * MB, xv[j]);
      } else {
#pragma unroll
        for (int v = 0; v < MB; ++v) a[j][v] = xv[j][v] = 0.0f;
      }
    }
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
      for (int v = 0; v < MB; ++v) ax = fmaf(a[j][v], xv[j][v], ax);
  }
  return ax;
}

template <int MB>
__global__ void __launch_bounds__(32 * MB) k_chebr(int nc, const int* __restrict__ rowptr, const int* __restrict__ col,
                                                   const float* __restrict__ aval, const float* __restrict__ dinv,
                                                   const float* __restrict__ b, const float* __restrict__ xin,
                                                   float* __restrict__ xout, float* __restrict__ d,
                                                   const float* __restrict__ lam, int l, int k, const int* done) {
  pdl_start();
  if (stop(done)) return;
  float c1, c2;
  cheb_tab(lam, l, k, c1, c2);
  __shared__ float rs[32 * MB];
  const int cl = threadIdx.x / MB, u = threadIdx.x - cl * MB;
  const int groups = (nc + 31) / 32;
  for (int g = blockIdx.x; g < groups; g += gridDim.x) {   // the same trip count in every thread of the block
    const int c = g * 32 + cl;
    const bool act = c < nc;
    const size_t i = (size_t)c * MB + u;
    float res = 0.0f, dv[MB];
    if (act) {
      ld_seg<MB>(dinv + i * MB, dv);
      res = b[i] - row_ax_u<MB>(c, u, rowptr, col, aval, xin);
    }
    rs[threadIdx.x] = res;
    __syncthreads();
    if (act) {
      float s = 0.0f;
#pragma unroll
      for (int v = 0; v < MB; ++v) s = fmaf(dv[v], rs[cl * MB + v], s);
      const float dn = (k == 0 ? 0.0f : c1 * d[i]) + c2 * s;
      d[i] = dn;
      xout[i] = xin[i] + dn;
    }
    __syncthreads();
  }
}

template <int MB>
__global__ void __launch_bounds__(32 * MB) k_resr(int nc, const int* __restrict__ rowptr, const int* __restrict__ col,
                                                  const float* __restrict__ aval, const float* __restrict__ b,
                                                  const float* __restrict__ x, float* __restrict__ res,
                                                  const int* done) {
  pdl_start();
  if (stop(done)) return;
  const long rows = (long)nc * MB;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i / MB), u = (int)(i - (long)c * MB);
    res[i] = b[i] - row_ax_u<MB>(c, u, rowptr, col, aval, x);
  }
}

// Level-0 restriction with MB modes per aggregate (FP32 or BF16 transfers): restr_body's work split and order (one
// warp per aggregate, a lane per child, children t and t + 32 together), with the child's MB transfer entries read
// by vector loads and the aggregate's block-inverse row (for the fused first smoothing step) requested before the
// products. Same sums in the same order, so the same values as the generic kernel.
template <class PT, int MB>
__global__ void k_restr0(const float* __restrict__ res, const PT* __restrict__ P, const int* __restrict__ ch_off,
                         const int* __restrict__ ch, int ncc, float* __restrict__ bc, const float* __restrict__ dinvc,
                         float* __restrict__ xc, float* __restrict__ dc, const float* __restrict__ lam, int first,
                         const int* done) {
  pdl_start();
  if (stop(done)) return;
  float c1 = 0.0f, c2 = 0.0f;
  if (first) cheb_tab(lam, 1, 0, c1, c2);
  const int lane = threadIdx.x & 31;
  for (int A = gwarp(); A < ncc; A += nwarps()) {
    float dv[MB];
    if (first && lane < MB) ld_seg<MB>(dinvc + ((size_t)A * MB + lane) * MB, dv);
    float acc[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) acc[j] = 0.0f;
    const int t1 = ch_off[A + 1];
    for (int t = ch_off[A] + lane; t < t1; t += 64) {
      const bool two = t + 32 < t1;
      const int ca = ch[t], cb = two ? ch[t + 32] : ca;
      const float ra = res[ca], rb = res[cb];
      float Pa[MB], Pb[MB];
      ld_seg<MB>(P + (size_t)ca * MB, Pa);
      ld_seg<MB>(P + (size_t)cb * MB, Pb);
#pragma unroll
      for (int j = 0; j < MB; ++j) acc[j] = fmaf(Pa[j], ra, acc[j]);
      if (two) {
#pragma unroll
        for (int j = 0; j < MB; ++j) acc[j] = fmaf(Pb[j], rb, acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < MB; ++j) acc[j] = warp_sum(acc[j]);
    if (lane < MB) {
      float bj = 0.0f;
#pragma unroll
      for (int j = 0; j < MB; ++j)
        if (j == lane) bj = acc[j];
      bc[(size_t)A * MB + lane] = bj;
      if (first) {
        float s = 0.0f;
#pragma unroll
        for (int v = 0; v < MB; ++v) s = fmaf(dv[v], acc[v], s);
        const float dn = c2 * s;
        dc[(size_t)A * MB + lane] = dn;
        xc[(size_t)A * MB + lane] = dn;
      }
    }
  }
}

// The small levels of one V-cycle in one launch of one thread block, out of shared memory: from the restriction of
// level t-1's residual (W.d[t-1], global) to the prolongation into level t-1 (W.x[t-1][cur_prev], global), the
// smoothing, residuals and transfers of levels t .. C-1 and the coarsest solve run as phases separated by
// __syncthreads on copies of their matrices, transfers and vectors held in shared memory, instead of one dependent
// kernel (a few L2 round trips) per phase. The copy-in is one pass of 16-byte loads, eight in flight per thread, from
// the table's copy list (every source array is allocated in whole 16-byte units). The phases are the bodies of the
// per-level kernels with the same work split per cell and the same order of operations, so the result does not depend
// on which form ran.
template <class PT>
__global__ void __launch_bounds__(kTailThreads, 1) k_small(const MgTailTab* __restrict__ Tg, int cur_prev) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ MgTailTab T_;   // the table itself, read by every phase
  static_assert(sizeof(MgTailTab) % 4 == 0, "table copied in words");
  pdl_start();
  for (int i = threadIdx.x; i < (int)(sizeof(MgTailTab) / 4); i += kTailThreads)
    ((int*)&T_)[i] = __ldg((const int*)Tg + i);
  __syncthreads();
  const MgTailTab* T = &T_;
  constexpr int v = std::is_same_v<PT, float> ? 0 : 1;
  {
    const int nch = T->nchunks[v], ncp = T->ncopies[v];
    for (int i0 = threadIdx.x; i0 < nch; i0 += kTailThreads * 8) {
      float4 buf[8];
      unsigned dst[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * kTailThreads;
        if (i < nch) {
          int lo = 0, hi = ncp - 1;   // last entry whose first chunk is <= i
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (T->cp[v][mid].c0 <= (unsigned)i) lo = mid;
            else hi = mid - 1;
          }
          const MgTailCopy& e = T->cp[v][lo];
          buf[u] = __ldg((const float4*)e.src + (i - e.c0));
          dst[u] = e.dst + 16u * (i - e.c0);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * kTailThreads < nch) *(float4*)(sm + dst[u]) = buf[u];
    }
  }
  __syncthreads();
  const MgDev& M = T->M;
  const int t = T->t, C = M.L - 1;
  const int w0 = threadIdx.x >> 5, nw = kTailThreads / 32;
  const int i0 = threadIdx.x, ni = kTailThreads;
  auto F32 = [&](unsigned off) { return (float*)(sm + off); };
  auto I32 = [&](unsigned off) { return (const int*)(sm + off); };
  auto PL = [&](int l) { return (const PT*)(sm + T->o_P[l]); };
  // buffer of level l's iterate: x[l][0] after the restriction (first step fused), then each Chebyshev step moves
  // it to the other buffer; the coarsest solve writes x[C][0]
  constexpr int kDown = (kMgDegCoarse - 1) & 1, kUp = (2 * kMgDegCoarse - 1) & 1;
  const float* coef = F32(T->o_coef);
  float c1, c2 = 0.0f;
  if (t < C) cheb_tab(coef, t, 0, c1, c2);
  restr_body<PT, false>(w0, nw, M.mb[t - 1], T->d[t - 1], PL(t - 1), I32(T->o_choff[t - 1]), I32(T->o_ch[t - 1]),
                        M.nc[t], M.mb[t], F32(T->o_b[t]), F32(T->o_dinv[t]), F32(T->o_x[t][0]), F32(T->o_d[t]), c2,
                        t < C ? 1 : 0);
  __syncthreads();
  for (int l = t; l < C; ++l) {
    const int *rp = I32(T->o_rowptr[l]), *cl = I32(T->o_col[l]);
    const float *av = F32(T->o_aval[l]), *di = F32(T->o_dinv[l]);
    float *xb[2] = {F32(T->o_x[l][0]), F32(T->o_x[l][1])}, *bl = F32(T->o_b[l]), *dl = F32(T->o_d[l]);
    for (int k = 1; k < kMgDegCoarse; ++k) {
      cheb_tab(coef, l, k, c1, c2);
      MG_MB_SWITCH(M.mb[l], (chebl_body<MB, false>(w0, nw, M.nc[l], rp, cl, av, di, bl, xb[(k - 1) & 1], xb[k & 1],
                                                   dl, c1, c2, k)));
      __syncthreads();
    }
    MG_MB_SWITCH(M.mb[l], (resl_body<MB, false>(w0, nw, M.nc[l], rp, cl, av, bl, xb[kDown], dl)));
    __syncthreads();
    const int first = l + 1 < C ? 1 : 0;
    c2 = 0.0f;
    if (first) cheb_tab(coef, l + 1, 0, c1, c2);
    restr_body<PT, false>(w0, nw, M.mb[l], dl, PL(l), I32(T->o_choff[l]), I32(T->o_ch[l]), M.nc[l + 1],
                          M.mb[l + 1], F32(T->o_b[l + 1]), F32(T->o_dinv[l + 1]), F32(T->o_x[l + 1][0]),
                          F32(T->o_d[l + 1]), c2, first);
    __syncthreads();
  }
  coarse_solve_body<false>(i0, ni, M.nc[C] * M.mb[C], F32(T->o_cinv), F32(T->o_b[C]), F32(T->o_x[C][0]));
  __syncthreads();
  for (int l = C - 1; l >= t; --l) {
    const int *rp = I32(T->o_rowptr[l]), *cl = I32(T->o_col[l]);
    const float *av = F32(T->o_aval[l]), *di = F32(T->o_dinv[l]);
    float *xb[2] = {F32(T->o_x[l][0]), F32(T->o_x[l][1])}, *bl = F32(T->o_b[l]), *dl = F32(T->o_d[l]);
    prol_body<PT, false>(i0, ni, M.nc[l], M.mb[l], M.mb[l + 1], PL(l), I32(T->o_agg[l]),
                         F32(T->o_x[l + 1][l + 1 == C ? 0 : kUp]), xb[kDown]);
    __syncthreads();
    for (int k = 0; k < kMgDegCoarse; ++k) {
      cheb_tab(coef, l, k, c1, c2);
      MG_MB_SWITCH(M.mb[l], (chebl_body<MB, false>(w0, nw, M.nc[l], rp, cl, av, di, bl, xb[(kDown + k) & 1],
                                                   xb[(kDown + k + 1) & 1], dl, c1, c2, k)));
      __syncthreads();
    }
  }
  prol_body<PT, false>(i0, ni, M.nc[t - 1], M.mb[t - 1], M.mb[t], PL(t - 1), I32(T->o_agg[t - 1]),
                       F32(T->o_x[t][t == C ? 0 : kUp]), T->x[t - 1][cur_prev]);
}

// ---------------------------------------------------------------------------------------------------------------
// Krylov kernels (FP64 outer iteration)

// A v with the frozen FP64 matrix (diagT, Tval) at cell K, v of type T.
template <class T>
__device__ __forceinline__ double amul(const FineDev& F, const double* __restrict__ Tval,
                                       const double* __restrict__ diagT, const T* __restrict__ v, int K) {
  const int w = F.sell_w[K >> 5];
  int e = F.sell_off[K >> 5] + (K & 31);
  double s = diagT[K] * (double)v[K];
  for (int j = 0; j < w; ++j, e += 32) s = fma(-Tval[e], (double)v[F.nbr[e]], s);
  return s;
}

// Fused first pre-smoothing step of level 0 for the FP32 right-hand side r32: x0 = D^-1 r32 / theta, d0 = x0.
__device__ __forceinline__ void first_step0(int K, float r32, const float* __restrict__ a0dinv, float c2,
                                            float* __restrict__ x0, float* __restrict__ d0) {
  const float dn = c2 * a0dinv[K] * r32;
  x0[K] = dn;
  d0[K] = dn;
}

// PCG start: x = 0, r = bscale b, r32 = r, first smoothing step, rr0 = ||S r||^2 (S = diag(A)^-1/2).
__global__ void k_pcg_init(int N, const double* __restrict__ b, double bscale, const double* __restrict__ diagT,
                           double* __restrict__ x, double* __restrict__ r, float* __restrict__ r32,
                           const float* __restrict__ a0dinv, float* __restrict__ x0, float* __restrict__ d0,
                           const float* __restrict__ lam, double* part, MgScal* sc) {
  pdl_start();
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  double v[1] = {0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    const double ri = bscale * b[K];
    x[K] = 0.0;
    r[K] = ri;
    r32[K] = (float)ri;
    first_step0(K, (float)ri, a0dinv, c2, x0, d0);
    v[0] = fma(ri * ri, (double)a0dinv[K], v[0]);   // ||S r||^2 with S^2 = 1 / A_KK
  }
  __shared__ double out[1];
  if (reduce_last<1>(v, part, &sc->cnt[0], out) && threadIdx.x == 0) {
    sc->rr0 = out[0];
    sc->rr = out[0];
    sc->it = 0;
    sc->done = !(out[0] > 0.0) ? 1 : 0;
    sc->bad = isfinite(out[0]) ? 0 : 1;
    sc->rz = 0.0;
  }
}

// p = z + beta p, q = A z + beta q (= A p), alpha = rz / (p, q); z is kept as z_old for the next beta.
__global__ void k_pcg_pq(FineDev F, const double* __restrict__ Tval, const double* __restrict__ diagT,
                         const float* __restrict__ z, float* __restrict__ zold, double* __restrict__ p,
                         double* __restrict__ q, double* part, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done)) return;
  const double beta = sc->beta;
  const bool first = sc->it == 0;
  double v[1] = {0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    const double az = amul<float>(F, Tval, diagT, z, K);
    const double pk = first ? (double)z[K] : fma(beta, p[K], (double)z[K]);
    const double qk = first ? az : fma(beta, q[K], az);
    p[K] = pk;
    q[K] = qk;
    zold[K] = z[K];
    v[0] = fma(pk, qk, v[0]);
  }
  __shared__ double out[1];
  if (reduce_last<1>(v, part, &sc->cnt[2], out) && threadIdx.x == 0) sc->alpha = sc->rz / out[0];
}

// x += alpha p, r -= alpha q, r32 = r with the first smoothing step of the next V-cycle; ||S r||^2 decides: the
// iteration stops (conditional value 0) at ||S r||^2 <= tol^2 ||S r_0||^2, at maxit, or on a non-finite value.
__global__ void k_pcg_update(int N, const double* __restrict__ p, const double* __restrict__ q,
                             const double* __restrict__ diagT, double* __restrict__ x, double* __restrict__ r,
                             float* __restrict__ r32, const float* __restrict__ a0dinv, float* __restrict__ x0,
                             float* __restrict__ d0, const float* __restrict__ lam, double* part, MgScal* sc,
                             cudaGraphConditionalHandle h) {
  pdl_start();
  if (stop(&sc->done)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0);
    return;
  }
  const double alpha = sc->alpha;
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  double v[1] = {0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    x[K] = fma(alpha, p[K], x[K]);
    const double ri = fma(-alpha, q[K], r[K]);
    r[K] = ri;
    r32[K] = (float)ri;
    first_step0(K, (float)ri, a0dinv, c2, x0, d0);
    v[0] = fma(ri * ri, (double)a0dinv[K], v[0]);   // ||S r||^2 with S^2 = 1 / A_KK
  }
  __shared__ double out[1];
  if (reduce_last<1>(v, part, &sc->cnt[3], out) && threadIdx.x == 0) {
    sc->rr = out[0];
    sc->it += 1;
    const bool fin = isfinite(out[0]) && isfinite(alpha);
    if (!fin) sc->bad = 1;
    const int d = (!fin || out[0] <= sc->tol2 * sc->rr0 || sc->it >= sc->maxit) ? 1 : 0;
    sc->done = d;
    cudaGraphSetConditional(h, d ? 0 : 1);
  }
}

// ---- BiCGStab (right-preconditioned) for J dx = bscale b with the Newton Jacobian (jd diagonal, Joff SELL) ------
template <class T>
__device__ __forceinline__ double jmul(const FineDev& F, const double* __restrict__ Joff,
                                       const double* __restrict__ jd, const T* __restrict__ v, int K) {
  const int w = F.sell_w[K >> 5];
  int e = F.sell_off[K >> 5] + (K & 31);
  double s = jd[K] * (double)v[K];
  for (int j = 0; j < w; ++j, e += 32) s = fma(Joff[e], (double)v[F.nbr[e]], s);
  return s;
}

// start: x = 0, r = rh = p = bscale b, rho = (rh, r), rr0 = ||W r||^2 (W the Jacobi weights' square roots);
// r32 = p for the first V-cycle (p^ = B p).
__global__ void k_bicg_init(int N, const double* __restrict__ b, double bscale, const double* __restrict__ wgt,
                            double* __restrict__ x, double* __restrict__ r, double* __restrict__ rh,
                            double* __restrict__ p, float* __restrict__ r32, const float* __restrict__ a0dinv,
                            float* __restrict__ x0, float* __restrict__ d0, const float* __restrict__ lam,
                            double* part, MgScal* sc) {
  pdl_start();
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  double v[2] = {0.0, 0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    const double ri = bscale * b[K];
    x[K] = 0.0;
    r[K] = ri;
    rh[K] = ri;
    p[K] = ri;
    r32[K] = (float)ri;
    first_step0(K, (float)ri, a0dinv, c2, x0, d0);
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(ri * ri, wgt[K], v[1]);
  }
  __shared__ double out[2];
  if (reduce_last<2>(v, part, &sc->cnt[0], out) && threadIdx.x == 0) {
    sc->rho = out[0];
    sc->rr0 = out[1];
    sc->rr = out[1];
    sc->it = 0;
    sc->done = !(out[1] > 0.0) ? 1 : 0;
    sc->bad = isfinite(out[1]) ? 0 : 1;
  }
}

// v = J p^ (p^ = B p from the V-cycle, kept in FP64 in pp); alpha = rho / (rh, v); s = r - alpha v, r32 = s with the
// first smoothing step of the next V-cycle (s^ = B s).
__global__ void k_bicg_v(FineDev F, const double* __restrict__ Joff, const double* __restrict__ jd,
                         const float* __restrict__ zp, double* __restrict__ pp, double* __restrict__ v,
                         const double* __restrict__ rh, double* part, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done)) return;
  double a[1] = {0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    pp[K] = (double)zp[K];
    const double vk = jmul<float>(F, Joff, jd, zp, K);
    v[K] = vk;
    a[0] = fma(rh[K], vk, a[0]);
  }
  __shared__ double out[1];
  if (reduce_last<1>(a, part, &sc->cnt[1], out) && threadIdx.x == 0) sc->alpha = sc->rho / out[0];
}
__global__ void k_bicg_s(int N, const double* __restrict__ r, const double* __restrict__ v, double* __restrict__ s,
                         float* __restrict__ r32, const float* __restrict__ a0dinv, float* __restrict__ x0,
                         float* __restrict__ d0, const float* __restrict__ lam, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done)) return;
  const double alpha = sc->alpha;
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    const double sk = fma(-alpha, v[K], r[K]);
    s[K] = sk;
    r32[K] = (float)sk;
    first_step0(K, (float)sk, a0dinv, c2, x0, d0);
  }
}
// t = J s^ (s^ = B s from the V-cycle), omega = (t, s) / (t, t).
__global__ void k_bicg_t(FineDev F, const double* __restrict__ Joff, const double* __restrict__ jd,
                         const float* __restrict__ zs, const double* __restrict__ s, double* __restrict__ t,
                         double* part, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done)) return;
  double a[2] = {0.0, 0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < F.N; K += gridDim.x * blockDim.x) {
    const double tk = jmul<float>(F, Joff, jd, zs, K);
    t[K] = tk;
    a[0] = fma(tk, s[K], a[0]);
    a[1] = fma(tk, tk, a[1]);
  }
  __shared__ double out[2];
  if (reduce_last<2>(a, part, &sc->cnt[2], out) && threadIdx.x == 0) sc->omega = out[1] != 0.0 ? out[0] / out[1] : 0.0;
}
// x += alpha p^ + omega s^, r = s - omega t, rho_new = (rh, r), ||W r||^2; beta = (rho_new / rho)(alpha / omega).
__global__ void k_bicg_x(int N, const double* __restrict__ pp, const float* __restrict__ zs,
                         const double* __restrict__ s, const double* __restrict__ t, const double* __restrict__ rh,
                         const double* __restrict__ wgt, double* __restrict__ x, double* __restrict__ r, double* part,
                         MgScal* sc, cudaGraphConditionalHandle h) {
  pdl_start();
  if (stop(&sc->done)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0);
    return;
  }
  const double alpha = sc->alpha, omega = sc->omega;
  double a[2] = {0.0, 0.0};
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    x[K] = fma(omega, (double)zs[K], fma(alpha, pp[K], x[K]));
    const double rk = fma(-omega, t[K], s[K]);
    r[K] = rk;
    a[0] = fma(rh[K], rk, a[0]);
    a[1] = fma(rk * rk, wgt[K], a[1]);
  }
  __shared__ double out[2];
  if (reduce_last<2>(a, part, &sc->cnt[3], out) && threadIdx.x == 0) {
    sc->rr = out[1];
    sc->it += 1;
    const bool fin = isfinite(out[1]) && isfinite(alpha) && isfinite(omega);
    if (!fin) sc->bad = 1;
    const bool breakdown = omega == 0.0 || sc->rho == 0.0;
    sc->beta = breakdown ? 0.0 : (out[0] / sc->rho) * (alpha / omega);
    sc->rho = out[0];
    const int d = (!fin || breakdown || out[1] <= sc->tol2 * sc->rr0 || sc->it >= sc->maxit) ? 1 : 0;
    sc->done = d;
    cudaGraphSetConditional(h, d ? 0 : 1);
  }
}
// p = r + beta (p - omega v), r32 = p with the first smoothing step of the next V-cycle; on the first iteration the
// start has set p = r and that step already.
__global__ void k_bicg_p(int N, const double* __restrict__ r, const double* __restrict__ v, double* __restrict__ p,
                         float* __restrict__ r32, const float* __restrict__ a0dinv, float* __restrict__ x0,
                         float* __restrict__ d0, const float* __restrict__ lam, MgScal* sc) {
  pdl_start();
  if (stop(&sc->done) || sc->it == 0) return;
  const double beta = sc->beta, omega = sc->omega;
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    const double pk = fma(beta, fma(-omega, v[K], p[K]), r[K]);
    p[K] = pk;
    r32[K] = (float)pk;
    first_step0(K, (float)pk, a0dinv, c2, x0, d0);
  }
}

// z (FP32) -> out (FP64), and the start of a single application: r32 = b, first smoothing step.
__global__ void k_apply_in(int N, const double* __restrict__ b, float* __restrict__ r32,
                           const float* __restrict__ a0dinv, float* __restrict__ x0, float* __restrict__ d0,
                           const float* __restrict__ lam) {
  pdl_start();
  float c1, c2;
  cheb_tab(lam, 0, 0, c1, c2);
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) {
    r32[K] = (float)b[K];
    first_step0(K, (float)b[K], a0dinv, c2, x0, d0);
  }
}
__global__ void k_apply_out(int N, const float* __restrict__ z, double* __restrict__ out) {
  pdl_start();
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < N; K += gridDim.x * blockDim.x) out[K] = (double)z[K];
}

}  // namespace

// ---------------------------------------------------------------------------------------------------------------
// host: static structure

int mg_levels_for(const Hierarchy& H) {
  for (int L = 2; L <= (int)H.levels.size() && L <= kMgMaxLevels; ++L) {
    const Level& C = H.levels[L - 1];
    int mb = 0;
    for (int c = 0; c < C.n_cells; ++c) mb = std::max(mb, C.m[c]);
    if ((long)C.n_cells * mb <= kMgMaxCoarse) return L;
  }
  return 0;
}

bool mg_build_host(const FineMesh& fm, const Hierarchy& H, int levels, MgHost& M, std::string& err) {
  if (levels < 2 || levels > (int)H.levels.size() || levels > kMgMaxLevels) {
    err = "multigrid preconditioner: bad number of levels";
    return false;
  }
  const int N = fm.n_cells;
  M.L = levels;
  M.N = N;
  M.nc[0] = N;
  M.mb[0] = 1;
  for (int l = 1; l < levels; ++l) {
    const Level& Lv = H.levels[l];
    M.nc[l] = Lv.n_cells;
    int mb = 1;
    for (int c = 0; c < Lv.n_cells; ++c) mb = std::max(mb, Lv.m[c]);
    if (mb > kMaxM) {
      err = "multigrid preconditioner: more than 8 modes per cell";
      return false;
    }
    M.mb[l] = mb;
    M.mcnt[l] = Lv.m;
  }
  if ((long)M.nc[levels - 1] * M.mb[levels - 1] > kMgMaxCoarse) {
    err = "multigrid preconditioner: the coarsest level has more than " + std::to_string(kMgMaxCoarse) +
          " unknowns";
    return false;
  }
  // fine SELL positions of each interior face from its first cell (the layout of the residual kernel), and the
  // Dirichlet entry of each Dirichlet face
  std::vector<int> deg(N, 0), dcount(N, 0), face_pos(fm.n_faces, -1), dir_pos(fm.n_faces, -1);
  for (int f = 0; f < fm.n_faces; ++f) {
    if (fm.bc[f] == 0) {
      face_pos[f] = deg[fm.fk[f]];
      ++deg[fm.fk[f]];
      ++deg[fm.fl[f]];
    } else if (fm.bc[f] == 1) {
      dir_pos[f] = dcount[fm.fk[f]]++;
    }
  }
  const int nsl = (N + 31) / 32;
  std::vector<long> soff(nsl + 1, 0);
  for (int s = 0; s < nsl; ++s) {
    int w = 0;
    for (int K = 32 * s; K < std::min(N, 32 * s + 32); ++K) w = std::max(w, deg[K]);
    soff[s + 1] = soff[s] + 32L * w;
  }
  std::vector<int> doff(N + 1, 0);
  for (int K = 0; K < N; ++K) doff[K + 1] = doff[K] + dcount[K];
  // transfers (padded) and children
  for (int l = 0; l + 1 < levels; ++l) {
    const Transfer& T = H.transfers[l];
    const Level& Lc = H.levels[l + 1];
    const int mbf = M.mb[l], mbc = M.mb[l + 1];
    const int ncf = M.nc[l];
    M.agg[l] = T.agg_of;
    M.ch_off[l] = T.agg_off;
    M.ch[l] = T.agg_cells;
    M.P[l].assign((size_t)ncf * mbf * mbc, 0.0f);
    const Level& Lf = H.levels[l];
    for (int a = 0; a < Lc.n_cells; ++a) {
      const int ma = Lc.m[a];
      int t = 0;
      for (int k = T.agg_off[a]; k < T.agg_off[a + 1]; ++k) {
        const int c = T.agg_cells[k];
        const int mc = l == 0 ? 1 : Lf.m[c];
        for (int u = 0; u < mc; ++u, ++t)
          for (int j = 0; j < ma; ++j)
            M.P[l][((size_t)c * mbf + u) * mbc + j] = (float)T.Pblk[T.pblk_off[a] + (size_t)t * ma + j];
      }
    }
  }
  // level 1: block pattern and contributions from the fine faces
  {
    const std::vector<int>& agg = H.transfers[0].agg_of;
    const int nc = M.nc[1];
    std::vector<std::map<int, std::vector<int4>>> rows(nc);
    for (int a = 0; a < nc; ++a) rows[a][a];
    for (int f = 0; f < fm.n_faces; ++f) {
      if (fm.bc[f] == 0) {
        const int K = fm.fk[f], Lc = fm.fl[f];
        const int e = (int)(soff[K >> 5] + 32L * face_pos[f] + (K & 31));
        const int a = agg[K], b = agg[Lc];
        if (a == b) {
          rows[a][a].push_back(make_int4(K, Lc, e, 0));
        } else {
          rows[a][a].push_back(make_int4(K, K, e, 1));
          rows[b][b].push_back(make_int4(Lc, Lc, e, 1));
          rows[a][b].push_back(make_int4(K, Lc, e, 2));
          rows[b][a].push_back(make_int4(Lc, K, e, 2));
        }
      } else if (fm.bc[f] == 1) {
        const int K = fm.fk[f];
        rows[agg[K]][agg[K]].push_back(make_int4(K, doff[K] + dir_pos[f], 0, 3));
      }
    }
    M.rowptr[1].assign(nc + 1, 0);
    M.dpos[1].assign(nc, 0);
    M.asm_off[1].push_back(0);
    for (int a = 0; a < nc; ++a) {
      for (auto& kv : rows[a]) {
        if (kv.first == a) M.dpos[1][a] = (int)M.col[1].size();
        M.col[1].push_back(kv.first);
        for (const int4& t : kv.second) M.asm_list[1].push_back(t);
        M.asm_off[1].push_back((int)M.asm_list[1].size());
      }
      M.rowptr[1][a + 1] = (int)M.col[1].size();
    }
    M.nblk[1] = (int)M.col[1].size();
  }
  // levels l >= 2: from the blocks of level l-1
  for (int l = 2; l < levels; ++l) {
    const std::vector<int>& agg = H.transfers[l - 1].agg_of;
    const int nc = M.nc[l], ncf = M.nc[l - 1];
    std::vector<std::map<int, std::vector<int4>>> rows(nc);
    for (int a = 0; a < nc; ++a) rows[a][a];
    for (int c = 0; c < ncf; ++c)
      for (int q = M.rowptr[l - 1][c]; q < M.rowptr[l - 1][c + 1]; ++q) {
        const int d = M.col[l - 1][q];
        rows[agg[c]][agg[d]].push_back(make_int4(q, c, d, 0));
      }
    M.rowptr[l].assign(nc + 1, 0);
    M.dpos[l].assign(nc, 0);
    M.asm_off[l].push_back(0);
    for (int a = 0; a < nc; ++a) {
      for (auto& kv : rows[a]) {
        if (kv.first == a) M.dpos[l][a] = (int)M.col[l].size();
        M.col[l].push_back(kv.first);
        for (const int4& t : kv.second) M.asm_list[l].push_back(t);
        M.asm_off[l].push_back((int)M.asm_list[l].size());
      }
      M.rowptr[l][a + 1] = (int)M.col[l].size();
    }
    M.nblk[l] = (int)M.col[l].size();
  }
  return true;
}

// ---------------------------------------------------------------------------------------------------------------
// host: enqueueing

namespace {

// Launches with programmatic stream serialization (each kernel starts its launch while its predecessor finishes;
// pdl_start() in every kernel orders the memory accesses). Launch errors surface through cudaGetLastError().
template <class... KArgs, class... Args>
void launchk(cudaStream_t st, int grid, int block, size_t smem, void (*k)(KArgs...), Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, (KArgs)args...);
}

inline int warps_grid(long warps) { return blocks_for(warps * 32, 65535); }
// blocks of the row-parallel block-level kernels: one per group of 32 cells
inline int row_grid(int nc) { return (int)std::min<long>((nc + 31) / 32, 1 << 20); }

// One Chebyshev step k, and the residual, of block level l: row-parallel from W.row_cells cells up, else one warp per
// cell.
void cheb_level(cudaStream_t st, const MgDev& M, const MgWork& W, int l, int k, int cur, const int* flag) {
  if (M.nc[l] >= W.row_cells) {
    MG_MB_SWITCH(M.mb[l], launchk(st, row_grid(M.nc[l]), 32 * MB, 0, k_chebr<MB>, M.nc[l], (const int*)M.rowptr[l],
                                  (const int*)M.col[l], (const float*)W.aval[l], (const float*)W.dinv[l],
                                  (const float*)W.b[l], (const float*)W.x[l][cur], W.x[l][1 - cur], W.d[l],
                                  (const float*)W.coef, l, k, flag));
  } else {
    MG_MB_SWITCH(M.mb[l], launchk(st, warps_grid(M.nc[l]), kT, 0, k_chebl<MB>, M.nc[l], (const int*)M.rowptr[l],
                                  (const int*)M.col[l], (const float*)W.aval[l], (const float*)W.dinv[l],
                                  (const float*)W.b[l], (const float*)W.x[l][cur], W.x[l][1 - cur], W.d[l],
                                  (const float*)W.coef, l, k, flag));
  }
}
void res_level(cudaStream_t st, const MgDev& M, const MgWork& W, int l, int cur, const int* flag) {
  if (M.nc[l] >= W.row_cells) {
    MG_MB_SWITCH(M.mb[l], launchk(st, row_grid(M.nc[l]), 32 * MB, 0, k_resr<MB>, M.nc[l], (const int*)M.rowptr[l],
                                  (const int*)M.col[l], (const float*)W.aval[l], (const float*)W.b[l],
                                  (const float*)W.x[l][cur], W.d[l], flag));
  } else {
    MG_MB_SWITCH(M.mb[l], launchk(st, warps_grid(M.nc[l]), kT, 0, k_resl<MB>, M.nc[l], (const int*)M.rowptr[l],
                                  (const int*)M.col[l], (const float*)W.aval[l], (const float*)W.b[l],
                                  (const float*)W.x[l][cur], W.d[l], flag));
  }
}

}  // namespace

void mg_enqueue_setup(cudaStream_t st, const MgDev& M, const FineDev& F, const MgWork& W, const double* Tval,
                      const double* diagT, const double* kap) {
  cudaMemsetAsync(W.lam, 0, kMgMaxLevels * sizeof(float), st);
  launchk(st, blocks_for(M.N, 4096), kT, 0, k_fine_vals, F, Tval, diagT, W.a0off, W.a0diag, W.a0dinv, W.lam);
  if (W.bf16) {
    MG_MB_SWITCH(M.mb[1], launchk(st, warps_grid(M.nblk[1]), kT, 0, k_asm1<MB, __nv_bfloat16>, M.nblk[1],
                                  (const int*)M.asm_off[1], (const int4*)M.asm_list[1],
                                  (const __nv_bfloat16*)M.Pb[0], Tval, kap, (const double*)F.dir_ups, W.aval[1]));
  } else {
    MG_MB_SWITCH(M.mb[1], launchk(st, warps_grid(M.nblk[1]), kT, 0, k_asm1<MB, float>, M.nblk[1],
                                  (const int*)M.asm_off[1], (const int4*)M.asm_list[1], (const float*)M.P[0], Tval,
                                  kap, (const double*)F.dir_ups, W.aval[1]));
  }
  launchk(st, blocks_for(M.nc[1]), kT, 0, k_pad_diag, M.nc[1], M.mb[1], (const int*)M.dpos[1],
          (const int*)M.mcnt[1], W.aval[1]);
  int n = 3;
  for (int l = 2; l < M.L; ++l) {
    if (W.bf16) {
      MG_MB_SWITCH(M.mb[l], launchk(st, warps_grid(M.nblk[l]), kT, 0, k_asml<MB, __nv_bfloat16>, M.nblk[l],
                                    M.mb[l - 1], (const int*)M.asm_off[l], (const int4*)M.asm_list[l],
                                    (const __nv_bfloat16*)M.Pb[l - 1], (const float*)W.aval[l - 1], W.aval[l]));
    } else {
      MG_MB_SWITCH(M.mb[l], launchk(st, warps_grid(M.nblk[l]), kT, 0, k_asml<MB, float>, M.nblk[l], M.mb[l - 1],
                                    (const int*)M.asm_off[l], (const int4*)M.asm_list[l], (const float*)M.P[l - 1],
                                    (const float*)W.aval[l - 1], W.aval[l]));
    }
    launchk(st, blocks_for(M.nc[l]), kT, 0, k_pad_diag, M.nc[l], M.mb[l], (const int*)M.dpos[l],
            (const int*)M.mcnt[l], W.aval[l]);
    n += 2;
  }
  for (int l = 1; l + 1 < M.L; ++l) {
    MG_MB_SWITCH(M.mb[l], launchk(st, blocks_for(M.nc[l]), 128, 0, k_block_inv<MB>, M.nc[l],
                                  (const int*)M.rowptr[l], (const int*)M.dpos[l], (const float*)W.aval[l], W.dinv[l],
                                  W.lam + l));
    ++n;
  }
  launchk(st, 1, 32, 0, k_cheb_table, (const float*)W.lam, W.coef);
  ++n;
  const int C = M.L - 1, nco = M.nc[C] * M.mb[C];
  launchk(st, 1, 512, (size_t)(nco * nco + nco) * sizeof(double), k_coarse_inv, M.nc[C], M.mb[C],
          (const int*)M.rowptr[C], (const int*)M.col[C], (const float*)W.aval[C], W.cinv);
  count_launch(n + 1);
}

namespace {

// Shared-memory layout of the small levels from t on (byte offsets, every array in whole 16-byte units); returns the
// total. P slots are sized for FP32 (BF16 transfers use half of theirs).
size_t small_layout(const MgDev& M, int t, MgTailTab* T) {
  const int C = M.L - 1;
  size_t off = 0;
  auto put = [&](unsigned* o, size_t bytes) {
    if (o) *o = (unsigned)off;
    off += (bytes + 15) & ~(size_t)15;
  };
  for (int l = t - 1; l < C; ++l) {   // transfers l -> l+1
    put(T ? &T->o_P[l] : nullptr, (size_t)M.nc[l] * M.mb[l] * M.mb[l + 1] * 4);
    put(T ? &T->o_choff[l] : nullptr, ((size_t)M.nc[l + 1] + 1) * 4);
    put(T ? &T->o_ch[l] : nullptr, (size_t)M.nc[l] * 4);
    put(T ? &T->o_agg[l] : nullptr, (size_t)M.nc[l] * 4);
  }
  for (int l = t; l <= C; ++l) {
    const size_t n = (size_t)M.nc[l] * M.mb[l], mm = (size_t)M.mb[l] * M.mb[l];
    put(T ? &T->o_b[l] : nullptr, n * 4);
    put(T ? &T->o_x[l][0] : nullptr, n * 4);
    if (l == C) break;
    put(T ? &T->o_rowptr[l] : nullptr, ((size_t)M.nc[l] + 1) * 4);
    put(T ? &T->o_col[l] : nullptr, (size_t)M.nblk[l] * 4);
    put(T ? &T->o_aval[l] : nullptr, (size_t)M.nblk[l] * mm * 4);
    put(T ? &T->o_dinv[l] : nullptr, (size_t)M.nc[l] * mm * 4);
    put(T ? &T->o_x[l][1] : nullptr, n * 4);
    put(T ? &T->o_d[l] : nullptr, n * 4);
  }
  const size_t nco = (size_t)M.nc[C] * M.mb[C];
  put(T ? &T->o_cinv : nullptr, nco * nco * 4);
  put(T ? &T->o_coef : nullptr, kMgMaxLevels * kMgMaxDeg * 2 * 4);
  return off;
}

}  // namespace

int mg_tail_level(const MgDev& M) {
  const int C = M.L - 1;
  for (int l = 2; l <= C; ++l)
    if (M.nc[l] <= kTailMaxCells && small_layout(M, l, nullptr) <= kTailSmem) return l;
  return 0;
}

void mg_fill_tail(cudaStream_t st, const MgDev& M, MgWork& W) {
  MgTailTab h;
  h.M = M;
  h.t = mg_tail_level(M);
  for (int l = 0; l < kMgMaxLevels; ++l) {
    h.d[l] = W.d[l];
    h.x[l][0] = W.x[l][0];
    h.x[l][1] = W.x[l][1];
  }
  W.tail_smem = 0;
  if (h.t > 0) {
    const int t = h.t, C = M.L - 1;
    W.tail_smem = small_layout(M, t, &h);
    // copy list: the static structure, the per-setup matrices and transfers (FP32 or BF16 P)
    for (int v = 0; v < 2; ++v) {
      unsigned c0 = 0;
      int n = 0;
      auto add = [&](const void* src, unsigned dst, size_t bytes) {
        const unsigned ch = (unsigned)((bytes + 15) / 16);
        if (ch == 0) return;
        h.cp[v][n++] = MgTailCopy{src, dst, c0};
        c0 += ch;
      };
      for (int l = t - 1; l < C; ++l) {
        const size_t np = (size_t)M.nc[l] * M.mb[l] * M.mb[l + 1];
        if (v == 0) add(M.P[l], h.o_P[l], np * 4);
        else add(M.Pb[l], h.o_P[l], np * 2);
        add(M.ch_off[l], h.o_choff[l], ((size_t)M.nc[l + 1] + 1) * 4);
        add(M.ch[l], h.o_ch[l], (size_t)M.nc[l] * 4);
        add(M.agg[l], h.o_agg[l], (size_t)M.nc[l] * 4);
      }
      for (int l = t; l < C; ++l) {
        const size_t mm = (size_t)M.mb[l] * M.mb[l];
        add(M.rowptr[l], h.o_rowptr[l], ((size_t)M.nc[l] + 1) * 4);
        add(M.col[l], h.o_col[l], (size_t)M.nblk[l] * 4);
        add(W.aval[l], h.o_aval[l], (size_t)M.nblk[l] * mm * 4);
        add(W.dinv[l], h.o_dinv[l], (size_t)M.nc[l] * mm * 4);
      }
      const size_t nco = (size_t)M.nc[C] * M.mb[C];
      add(W.cinv, h.o_cinv, nco * nco * 4);
      add(W.coef, h.o_coef, kMgMaxLevels * kMgMaxDeg * 2 * 4);
      h.ncopies[v] = n;
      h.nchunks[v] = (int)c0;
    }
  }
  // pageable source: the call returns once the table is staged, so h may go out of scope
  cudaMemcpyAsync(W.tail, &h, sizeof(MgTailTab), cudaMemcpyHostToDevice, st);
}

namespace {

template <class PT>
void launch_small(cudaStream_t st, const MgWork& W, int cur_prev) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = W.tail_smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_small<PT>, (const MgTailTab*)W.tail, cur_prev);
}

}  // namespace

// The V-cycle after the fused first step of level 0 (x[0][0], d[0] set from b[0]); returns the index of the level-0
// buffer that holds z. Levels from mg_tail_level on run in one launch of k_small.
int mg_enqueue_vcycle(cudaStream_t st, const MgDev& M, const FineDev& F, const MgWork& W, const int* flag,
                      bool cg_beta) {
  const int L = M.L, C = L - 1;
  const int tl = mg_tail_level(M);
  const int top = tl > 0 ? tl - 1 : C;   // levels 1 .. top-1 restrict with their own kernels
  int cur[kMgMaxLevels] = {0};
  const int g0 = blocks_for(M.N, W.grid0);
  // down: level-0 smoothing, residual into d[0] (dead until the post-smoothing rewrites it), restriction
  for (int k = 1; k < kMgDegFine; ++k) {
    launchk(st, g0, kT, 0, k_cheb0, F, (const float*)W.a0off, (const float*)W.a0diag, (const float*)W.a0dinv,
            (const float*)W.b[0], (const float*)W.x[0][cur[0]], W.x[0][1 - cur[0]], W.d[0], (const float*)W.coef, k,
            flag);
    cur[0] ^= 1;
  }
  launchk(st, g0, kT, 0, k_res0, F, (const float*)W.a0off, (const float*)W.a0diag, (const float*)W.b[0],
          (const float*)W.x[0][cur[0]], W.d[0], flag);
  if (W.bf16) {
    MG_MB_SWITCH(M.mb[1], launchk(st, warps_grid(M.nc[1]), kT, 0, k_restr0<__nv_bfloat16, MB>, (const float*)W.d[0],
                                  (const __nv_bfloat16*)M.Pb[0], (const int*)M.ch_off[0], (const int*)M.ch[0], M.nc[1],
                                  W.b[1], (const float*)W.dinv[1], W.x[1][0], W.d[1], (const float*)W.coef,
                                  C > 1 ? 1 : 0, flag));
  } else {
    MG_MB_SWITCH(M.mb[1], launchk(st, warps_grid(M.nc[1]), kT, 0, k_restr0<float, MB>, (const float*)W.d[0],
                                  (const float*)M.P[0], (const int*)M.ch_off[0], (const int*)M.ch[0], M.nc[1], W.b[1],
                                  (const float*)W.dinv[1], W.x[1][0], W.d[1], (const float*)W.coef, C > 1 ? 1 : 0,
                                  flag));
  }
  for (int l = 1; l < C && l <= top; ++l) {
    for (int k = 1; k < kMgDegCoarse; ++k) {
      cheb_level(st, M, W, l, k, cur[l], flag);
      cur[l] ^= 1;
    }
    res_level(st, M, W, l, cur[l], flag);
    if (l == top) break;   // the tail restricts from here
    if (W.bf16)
      launchk(st, warps_grid(M.nc[l + 1]), kT, 0, k_restr<__nv_bfloat16>, M.mb[l], (const float*)W.d[l],
              (const __nv_bfloat16*)M.Pb[l], (const int*)M.ch_off[l], (const int*)M.ch[l], M.nc[l + 1],
              M.mb[l + 1], W.b[l + 1], (const float*)W.dinv[l + 1], W.x[l + 1][0], W.d[l + 1],
              (const float*)W.coef, l + 1, l + 1 < C ? 1 : 0, flag);
    else
      launchk(st, warps_grid(M.nc[l + 1]), kT, 0, k_restr<float>, M.mb[l], (const float*)W.d[l],
              (const float*)M.P[l], (const int*)M.ch_off[l], (const int*)M.ch[l], M.nc[l + 1], M.mb[l + 1],
              W.b[l + 1], (const float*)W.dinv[l + 1], W.x[l + 1][0], W.d[l + 1], (const float*)W.coef, l + 1,
              l + 1 < C ? 1 : 0, flag);
  }
  if (tl > 0) {
    if (W.bf16)
      launch_small<__nv_bfloat16>(st, W, cur[tl - 1]);
    else
      launch_small<float>(st, W, cur[tl - 1]);
  } else {
    launchk(st, 1, kMgMaxCoarse, 0, k_coarse_solve, M.nc[C] * M.mb[C], (const float*)W.cinv, (const float*)W.b[C],
            W.x[C][0], flag);
  }
  // up
  for (int l = std::min(top, C - 1); l >= 1; --l) {
    if (l != top || tl == 0) {
      if (W.bf16)
        launchk(st, blocks_for((long)M.nc[l] * M.mb[l]), kT, 0, k_prol<__nv_bfloat16>, M.nc[l], M.mb[l],
                M.mb[l + 1], (const __nv_bfloat16*)M.Pb[l], (const int*)M.agg[l],
                (const float*)W.x[l + 1][cur[l + 1]], W.x[l][cur[l]], flag);
      else
        launchk(st, blocks_for((long)M.nc[l] * M.mb[l]), kT, 0, k_prol<float>, M.nc[l], M.mb[l], M.mb[l + 1],
                (const float*)M.P[l], (const int*)M.agg[l], (const float*)W.x[l + 1][cur[l + 1]], W.x[l][cur[l]],
                flag);
    }
    for (int k = 0; k < kMgDegCoarse; ++k) {
      cheb_level(st, M, W, l, k, cur[l], flag);
      cur[l] ^= 1;
    }
  }
  if (W.bf16)
    launchk(st, g0, kT, 0, k_pro0<__nv_bfloat16>, M.N, M.mb[1], (const __nv_bfloat16*)M.Pb[0],
            (const int*)M.agg[0], (const float*)W.x[1][cur[1]], W.x[0][cur[0]], flag);
  else
    launchk(st, g0, kT, 0, k_pro0<float>, M.N, M.mb[1], (const float*)M.P[0], (const int*)M.agg[0],
            (const float*)W.x[1][cur[1]], W.x[0][cur[0]], flag);
  for (int k = 0; k < kMgDegFine; ++k) {
    if (cg_beta && k + 1 == kMgDegFine)
      launchk(st, blocks_for(M.N, kMaxRedBlocks), kT, 0, k_cheb0_beta, F, (const float*)W.a0off,
              (const float*)W.a0diag, (const float*)W.a0dinv, (const float*)W.b[0], (const float*)W.x[0][cur[0]],
              W.x[0][1 - cur[0]], W.d[0], (const float*)W.coef, k, (const double*)W.kr, (const float*)W.z[0], W.part,
              W.sc);
    else
      launchk(st, g0, kT, 0, k_cheb0, F, (const float*)W.a0off, (const float*)W.a0diag, (const float*)W.a0dinv,
              (const float*)W.b[0], (const float*)W.x[0][cur[0]], W.x[0][1 - cur[0]], W.d[0], (const float*)W.coef,
              k, flag);
    cur[0] ^= 1;
  }
  return cur[0];
}

int mg_vcycle_kernels(const MgDev& M) {
  const int C = M.L - 1, tl = mg_tail_level(M);
  const int level0 = (kMgDegFine - 1) + 2 + 1 + kMgDegFine;   // smoothing, residual, restriction, prolongation
  if (tl == 0) return level0 + (C - 1) * (kMgDegCoarse + 1) + 1 + (C - 1) * (1 + kMgDegCoarse);
  // levels 1 .. tl-1 run their own kernels: down smoothing and residual, the restrictions between them, and on the
  // way up the prolongations between them and the smoothing; the tail is one more
  const int own = tl - 1;
  return level0 + 2 * own * kMgDegCoarse + 2 * (own - 1) + 1;
}

namespace {

// A graph with one conditional while node whose body is captured from `body(handle)`.
template <class Body>
cudaError_t capture_while(cudaStream_t st, Body&& body, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
      cudaGraph_t bg = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(st, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        body(h);
        cudaError_t e2 = cudaStreamEndCapture(st, &bg);
        e = e2 != cudaSuccess ? e2 : cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

template <class Body>
cudaError_t capture_plain(cudaStream_t st, Body&& body, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  body();
  e = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

}  // namespace

// Preconditioned CG for A dx = -b (b = W.kb, FP64; dx -> W.kx) as two graphs: out[0] the start (x = 0, r = -b with
// the first smoothing step of the first V-cycle), out[1] the conditional while loop over the iterations (V-cycle with
// beta in its last step, p and q, x and r with the convergence test). The tolerance and iteration cap are read from
// W.sc at run time.
cudaError_t mg_capture_pcg(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, const double* Tval,
                           const double* diagT, cudaGraphExec_t* out) {
  const int gr = blocks_for(M.N, kMaxRedBlocks);
  cudaError_t e = capture_plain(st, [&]() {
    launchk(st, gr, kT, 0, k_pcg_init, M.N, (const double*)W.kb, -1.0, diagT, W.kx, W.kr, W.b[0],
            (const float*)W.a0dinv, W.x[0][0], W.d[0], (const float*)W.coef, W.part, W.sc);
  }, &out[0]);
  if (e != cudaSuccess) return e;
  // the convergence test is the body's last kernel, so nothing runs after it; the V-cycle kernels need no stop flag
  // (they only write the preconditioner's scratch and z)
  return capture_while(st, [&](cudaGraphConditionalHandle h) {
    const float* z = W.x[0][mg_enqueue_vcycle(st, M, F, W, nullptr, true)];   // its last step gives beta
    launchk(st, gr, kT, 0, k_pcg_pq, F, Tval, diagT, z, W.z[0], W.kp, W.kq, W.part, W.sc);
    launchk(st, gr, kT, 0, k_pcg_update, M.N, (const double*)W.kp, (const double*)W.kq, diagT, W.kx, W.kr, W.b[0],
            (const float*)W.a0dinv, W.x[0][0], W.d[0], (const float*)W.coef, W.part, W.sc, h);
  }, &out[1]);
}

// Right-preconditioned BiCGStab for J dx = -b (J: jd diagonal, Joff off-diagonal in the SELL layout; b = W.kb;
// dx -> W.kx; stopping on ||W r|| with W^2 = wgt). out[0] the start (r, r^, p = r with the first smoothing step of
// p^ = B p), out[1] the loop: p (from the second iteration on), p^ = B p, v = J p^, s, s^ = B s, t = J s^, then x
// and r with the convergence test as the last kernel.
cudaError_t mg_capture_bicgstab(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, const double* jd,
                                const double* Joff, const double* wgt, cudaGraphExec_t* out) {
  const int gr = blocks_for(M.N, kMaxRedBlocks);
  cudaError_t e = capture_plain(st, [&]() {
    launchk(st, gr, kT, 0, k_bicg_init, M.N, (const double*)W.kb, -1.0, wgt, W.kx, W.kr, W.krh, W.kp, W.b[0],
            (const float*)W.a0dinv, W.x[0][0], W.d[0], (const float*)W.coef, W.part, W.sc);
  }, &out[0]);
  if (e != cudaSuccess) return e;
  return capture_while(st, [&](cudaGraphConditionalHandle h) {
    launchk(st, gr, kT, 0, k_bicg_p, M.N, (const double*)W.kr, (const double*)W.kv, W.kp, W.b[0],
            (const float*)W.a0dinv, W.x[0][0], W.d[0], (const float*)W.coef, W.sc);
    const int zp = mg_enqueue_vcycle(st, M, F, W, nullptr, false);
    launchk(st, gr, kT, 0, k_bicg_v, F, Joff, jd, (const float*)W.x[0][zp], W.kpp, W.kv, (const double*)W.krh,
            W.part, W.sc);
    launchk(st, gr, kT, 0, k_bicg_s, M.N, (const double*)W.kr, (const double*)W.kv, W.ks, W.b[0],
            (const float*)W.a0dinv, W.x[0][0], W.d[0], (const float*)W.coef, W.sc);
    const int zs = mg_enqueue_vcycle(st, M, F, W, nullptr, false);
    launchk(st, gr, kT, 0, k_bicg_t, F, Joff, jd, (const float*)W.x[0][zs], (const double*)W.ks, W.kt, W.part,
            W.sc);
    launchk(st, gr, kT, 0, k_bicg_x, M.N, (const double*)W.kpp, (const float*)W.x[0][zs], (const double*)W.ks,
            (const double*)W.kt, (const double*)W.krh, wgt, W.kx, W.kr, W.part, W.sc, h);
  }, &out[1]);
}

// One V-cycle z = B b for parity tests: b = W.kb (FP64) -> W.kx (FP64).
cudaError_t mg_capture_apply(cudaStream_t st, const MgDev& M, const FineDev& F, MgWork& W, cudaGraphExec_t* out) {
  return capture_plain(st, [&]() {
    const int g0 = blocks_for(M.N, W.grid0);
    launchk(st, g0, kT, 0, k_apply_in, M.N, (const double*)W.kb, W.b[0], (const float*)W.a0dinv, W.x[0][0], W.d[0],
            (const float*)W.coef);
    const int zi = mg_enqueue_vcycle(st, M, F, W, nullptr, false);
    launchk(st, g0, kT, 0, k_apply_out, M.N, (const float*)W.x[0][zi], W.kx);
  }, out);
}

void mg_set_smem_limits() {
  static const bool once = [] {   // thread-safe one-time initialisation
    cudaFuncSetAttribute(k_coarse_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (kMgMaxCoarse * kMgMaxCoarse + kMgMaxCoarse) * (int)sizeof(double));
    cudaFuncSetAttribute(k_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem);
    cudaFuncSetAttribute(k_small<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem);
    return true;
  }();
  (void)once;
}

}  // namespace nlmg
