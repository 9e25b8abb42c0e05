// Persistent (cooperative) kernels: one launch runs a whole level-0 linear solve (the Picard step's CG, the Newton
// step's BiCGStab) or whole coarse Picard steps (hybridized CG, clamp, Algorithm 1), with device-side scalars,
// decisions and convergence tests, so the iterations pay neither launch gaps nor host round trips.
//
// Grid-wide synchronisation uses a counter barrier whose wait is bounded: after ~2 s of spinning the
// kernel records an error flag and every block leaves. The launch goes through cudaLaunchCooperativeKernel with at
// most the co-resident number of blocks, so in a correct run every wait ends.
//
// Data written by one block and read by another inside the same launch (CG vectors, per-interface buffers) is read
// with ld.global.cg (L2, bypassing the non-coherent L1), after the barrier that orders the write.
//
// Reductions stay deterministic: each block writes one partial per value; after the barrier every block adds all
// partials in block order with the same fixed tree and derives the step lengths once (one thread per block), so all
// blocks take the same decisions from bit-identical scalars and a run is bitwise reproducible for a given grid.
#include <cmath>

#include "kernels.cuh"
#include "persist.cuh"

namespace nlmg {

namespace {

constexpr unsigned long long kSpinLimit = 1ull << 26;   // x ~32 ns sleeps ~ 2 s
constexpr int kPThreads = 512;                           // threads per block of the persistent kernels
constexpr int kMaxNV = 4;                                // values per block reduction at most
constexpr int kSmDoubles = kMaxNV * kPThreads;           // block-reduction scratch: one value per thread

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// The synchronisation state one thread of a persistent kernel carries: the launch's barrier words, the two
// buffers of per-block partial sums (used alternately by consecutive reductions), kSmDoubles doubles of shared
// memory and the number of reductions so far (the same in every block).
struct Grid {
  GridSync gs;
  double* partial;
  double* sm;
  unsigned seq;
};

// Bounded grid barrier with one atomic per block: every block adds 1 to gs.count except block 0, which adds
// 2^31 - (gridDim.x - 1), so the counter's top bit flips exactly when the last block arrives and its low bits return
// to 0 (barriers follow one another without a reset). Thread 0 arrives with an acquire-release atomic after
// __syncthreads (its release covers the block's earlier writes) and polls the counter with acquire loads until the
// top bit differs from the value it added to. Returns false (and sets *err) if the wait gave up after ~2 s.
__device__ __forceinline__ bool grid_barrier(Grid& g, unsigned long long spin_limit = kSpinLimit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    const unsigned old = atom_add_acq_rel_gpu(g.gs.count, inc);
    unsigned long long spins = 0;
    while (((ld_acquire_gpu(g.gs.count) ^ old) & 0x80000000u) == 0u) {
      __nanosleep(32);
      if ((++spins & 1023u) == 0 && (spins > spin_limit || *((volatile int*)g.gs.err) != 0)) {
        atomicExch(g.gs.err, 1);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Grid sums of NV values. The FP64 pipe of this part is narrow (about 1.7 FP64 operations per clock per SM), so the
// block sums spend as few FP64 lane operations as possible: every thread stores its NV values to shared memory and
// warp k (k < NV) adds value k of all threads -- 16 per lane in a fixed order with four accumulators, then a
// shuffle tree -- about 640 lane operations per value instead of 2,560 for a shuffle tree in every warp (measured:
// a three-value grid sum 8.8 us -> 4.8 us). The block sum goes to the partial buffer; after the barrier warp k adds
// value k of every block's partial in block order, so all blocks hold bit-identical sums; thread 0 then runs
// `post(o)`, which derives NX scalars from the sums (the CG step lengths) into o[NV..NV+NX-1] in shared memory, so
// each division is done once per block, not per thread. Consecutive reductions use the two partial buffers in
// turn: a block can only overwrite a buffer after every block has passed the next barrier, i.e. has finished
// reading it.
template <int NV, int NX = 0, class PostFn>
__device__ __forceinline__ bool grid_sum_x(Grid& g, double (&v)[NV + NX], PostFn&& post) {
  static_assert(NV >= 1 && NV <= kMaxNV, "grid_sum_x: the shared scratch holds kMaxNV values per thread");
  static_assert(kPThreads % 128 == 0 && kPThreads / 32 >= kMaxNV, "grid_sum_x: block shape");
  double* part = g.partial + (g.seq & 1u) * kPartStride;
  ++g.seq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) g.sm[k * kPThreads + threadIdx.x] = v[k];
  __syncthreads();
  if (warp < NV) {
    const double* s = g.sm + warp * kPThreads;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int j = lane; j < kPThreads; j += 128) {
      a0 += s[j];
      a1 += s[j + 32];
      a2 += s[j + 64];
      a3 += s[j + 96];
    }
    double a = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) part[blockIdx.x * NV + warp] = a;
  }
  if (!grid_barrier(g)) return false;
  __shared__ double o[NV + NX];
  if (warp < NV) {
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(&part[b * NV + warp]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) o[warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) post(o);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV + NX; ++k) v[k] = o[k];
  return true;
}

template <int NV>
__device__ __forceinline__ bool grid_sum(Grid& g, double (&v)[NV]) {
  return grid_sum_x<NV, 0>(g, v, [](double*) {});
}

// Max over the grid of one value per thread (exact, hence deterministic), by the same protocol.
__device__ __forceinline__ bool grid_max(Grid& g, double& v) {
  double* part = g.partial + (g.seq & 1u) * kPartStride;
  ++g.seq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double m = v;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if (lane == 0) g.sm[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bm = g.sm[0];
    for (int w = 1; w < nw; ++w) bm = fmax(bm, g.sm[w]);
    part[blockIdx.x] = bm;
  }
  if (!grid_barrier(g)) return false;
  double gm = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) gm = fmax(gm, __ldcg(&part[b]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) gm = fmax(gm, __shfl_down_sync(0xffffffffu, gm, off));
  if (lane == 0) g.sm[warp] = gm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bm = g.sm[0];
    for (int w = 1; w < nw; ++w) bm = fmax(bm, g.sm[w]);
    g.sm[32] = bm;
  }
  __syncthreads();
  v = g.sm[32];
  __syncthreads();
  return true;
}

#define GSTRIDE(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// ---- fine level: A dx = bscale * b with the frozen TPFA matrix --------------------------------------------------
// CG on the symmetrically Jacobi-scaled system (S A S) y = S bscale b, dx = S y, S = diag(A)^-1/2, so the scaled
// matrix has a unit diagonal and only its off-diagonal entries Ts (SELL-32 layout, type T) are read. T = double is
// the FP64 path; T = float runs the Krylov vectors and the matrix in FP32 inside the FP64 nonlinear iteration
// (per-thread partial sums of the dot products in FP32, block and grid sums in FP64). The matrix is applied to the residual r, which every iteration already
// materialises, and A p follows by recurrence (p = r + beta p, q = A r + beta q): no neighbour values have to be
// rebuilt and an iteration needs two grid barriers. The stopping test is on the scaled residual,
// ||S r|| <= tol ||S r_0|| (the r.z of Jacobi-preconditioned CG).
template <class T>
__global__ void __launch_bounds__(kPThreads) kp_fine_cg(FineDev F, const T* __restrict__ Ts,
                                                        const double* __restrict__ sdiag,
                                                        const double* __restrict__ b, double bscale,
                                                        double* __restrict__ dx, T* __restrict__ y,
                                                        T* __restrict__ r, T* __restrict__ p, T* __restrict__ q,
                                                        double* partial, GridSync gs, double tol, int maxit,
                                                        PcgResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  T t1 = (T)0;   // per-thread partial sums in T (a thread holds one or two cells), block and grid sums in FP64
  GSTRIDE(i, F.N) {
    const T ri = (T)(sdiag[i] * bscale * b[i]);
    y[i] = (T)0;
    r[i] = ri;
    t1 = fma(ri, ri, t1);
  }
  double a1[1] = {(double)t1};
  if (!grid_sum<1>(g, a1)) return;
  const double rr0 = a1[0];
  double rr = rr0;
  const double tol2 = tol * tol * rr0;
  T beta = (T)0;
  int it = 0;
  while (rr0 > 0.0 && rr > tol2 && it < maxit) {
    T tpq = (T)0;
    GSTRIDE(K, F.N) {
      const int s = K >> 5, lane = K & 31;
      const T rK = __ldcg(&r[K]);
      T acc = rK;
      const int w = F.sell_w[s];
      int e = F.sell_off[s] + lane;
      int j = 0;
      if (w <= 8) {
        int Ls[8];
        T Tv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < w) {
            Ls[u] = F.nbr[e + 32 * u];
            Tv[u] = Ts[e + 32 * u];
          }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < w) acc -= Tv[u] * __ldcg(&r[Ls[u]]);
        j = w;
      }
      for (e += 32 * j; j < w; ++j, e += 32) acc -= Ts[e] * __ldcg(&r[F.nbr[e]]);
      const T pK = it == 0 ? rK : rK + beta * p[K];
      const T qK = it == 0 ? acc : acc + beta * q[K];
      p[K] = pK;
      q[K] = qK;
      tpq = fma(pK, qK, tpq);
    }
    double pq[2] = {(double)tpq, 0.0};
    if (!grid_sum_x<1, 1>(g, pq, [&](double* o) { o[1] = o[0] != 0.0 ? rr / o[0] : 0.0; }))
      return;
    const double alpha_d = pq[1];
    const T alpha = (T)alpha_d;
    T trn = (T)0;
    GSTRIDE(i, F.N) {
      y[i] = alpha * p[i] + y[i];
      const T ri = r[i] - alpha * q[i];
      r[i] = ri;
      trn = fma(ri, ri, trn);
    }
    double rn[2] = {(double)trn, 0.0};
    if (!grid_sum_x<1, 1>(g, rn, [&](double* o) { o[1] = rr != 0.0 ? o[0] / rr : 0.0; }))
      return;
    beta = (T)rn[1];
    rr = rn[0];
    ++it;
    if (!(alpha_d != 0.0)) break;   // breakdown (p.Ap = 0): stop with the current iterate
  }
  GSTRIDE(i, F.N) dx[i] = sdiag[i] * (double)y[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = rr;
  }
}

// Pipelined CG (Ghysels and Vanroose) on the same scaled system: the dot products of an iteration are computed from
// vectors updated in the same pass as the matrix product, so one grid barrier per iteration both publishes the
// vector the next matrix product gathers and completes the reduction. Recurrences: n = A w, z = n + beta z,
// s = w + beta s, p = r + beta p, y += alpha p, r -= alpha s, w -= alpha z; gamma = (r, r), delta = (w, r). Used for
// loose tolerances (the recursively updated residual drifts from the true one at the 1e-10 level).
template <class T>
__device__ __forceinline__ T sell_apply(const FineDev& F, const T* __restrict__ Ts, const T* v, int K) {
  const int s = K >> 5, lane = K & 31;
  T acc = __ldcg(&v[K]);
  const int w = F.sell_w[s];
  int e = F.sell_off[s] + lane;
  int j = 0;
  if (w <= 8) {
    int Ls[8];
    T Tv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < w) {
        Ls[u] = F.nbr[e + 32 * u];
        Tv[u] = Ts[e + 32 * u];
      }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < w) acc -= Tv[u] * __ldcg(&v[Ls[u]]);
    j = w;
  }
  for (e += 32 * j; j < w; ++j, e += 32) acc -= Ts[e] * __ldcg(&v[F.nbr[e]]);
  return acc;
}

template <class T>
__global__ void __launch_bounds__(kPThreads) kp_fine_cg_pipe(FineDev F, const T* __restrict__ Ts,
                                                             const double* __restrict__ sdiag,
                                                             const double* __restrict__ b, double bscale,
                                                             double* __restrict__ dx, T* __restrict__ y,
                                                             T* __restrict__ r, T* wa, T* wb, T* __restrict__ z,
                                                             T* __restrict__ sv, T* __restrict__ p, double* partial,
                                                             GridSync gs, double tol, int maxit, PcgResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  GSTRIDE(i, F.N) {
    r[i] = (T)(sdiag[i] * bscale * b[i]);
    y[i] = z[i] = sv[i] = p[i] = (T)0;
  }
  if (!grid_barrier(g)) return;
  // a4 = {gamma, delta, beta, alpha}: the sums and, from the last block's thread 0, the step lengths of the next
  // iteration (beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old); first: 0, gamma / delta)
  double a4[4] = {0.0, 0.0, 0.0, 0.0};
  GSTRIDE(K, F.N) {
    const T wK = sell_apply<T>(F, Ts, r, K);
    wa[K] = wK;
    const double rK = (double)r[K];
    a4[0] = fma(rK, rK, a4[0]);
    a4[1] = fma((double)wK, rK, a4[1]);
  }
  if (!grid_sum_x<2, 2>(g, a4, [&](double* o) {
        o[2] = 0.0;
        o[3] = o[1] != 0.0 ? o[0] / o[1] : 0.0;
      }))
    return;
  double gamma = a4[0], beta_d = a4[2], alpha_d = a4[3];
  const double rr0 = gamma;
  const double tol2 = tol * tol * rr0;
  T* wc = wa;   // current w (read, neighbours gathered)
  T* wn = wb;   // next w (written)
  int it = 0;
  while (rr0 > 0.0 && gamma > tol2 && it < maxit) {
    if (!(alpha_d != 0.0)) break;
    const T alpha = (T)alpha_d, beta = (T)beta_d;
    double n4[4] = {0.0, 0.0, 0.0, 0.0};
    GSTRIDE(K, F.N) {
      const T nK = sell_apply<T>(F, Ts, wc, K);
      const T wK = wc[K];
      const T zK = nK + beta * z[K];
      const T sK = wK + beta * sv[K];
      const T pK = r[K] + beta * p[K];
      z[K] = zK;
      sv[K] = sK;
      p[K] = pK;
      y[K] += alpha * pK;
      const T rK = r[K] - alpha * sK;
      r[K] = rK;
      const T wN = wK - alpha * zK;
      wn[K] = wN;
      n4[0] = fma((double)rK, (double)rK, n4[0]);
      n4[1] = fma((double)wN, (double)rK, n4[1]);
    }
    if (!grid_sum_x<2, 2>(g, n4, [&](double* o) {
          const double g = o[0], d = o[1];
          const double bn = gamma != 0.0 ? g / gamma : 0.0;
          const double den = d - bn * g / alpha_d;
          o[2] = bn;
          o[3] = den != 0.0 ? g / den : 0.0;
        }))
      return;
    gamma = n4[0];
    beta_d = n4[2];
    alpha_d = n4[3];
    T* t = wc;
    wc = wn;
    wn = t;
    ++it;
  }
  GSTRIDE(i, F.N) dx[i] = sdiag[i] * (double)y[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = gamma;
  }
}

// Register-resident pipelined CG. A persistent thread owns the same cells (at most R of them: K = k0 + u * stride)
// for the whole solve, so y, r, p, s, z and w of its cells stay in FP64 registers; only w, which the neighbours
// gather, is written to memory (double-buffered, type TM) each iteration. Per iteration: n = A w from the published
// w, the recurrences of the pipelined CG above, the two dot products, one grid barrier. TM = double gives the FP64
// path (bitwise the memory-resident kernel on the same grid). (TM = float, an FP32 matrix product inside FP64
// recurrences, was measured to drift like the all-FP32 pipelined form and is not used.)
template <class TM, int R>
__global__ void __launch_bounds__(kPThreads) kp_fine_cg_reg(FineDev F, const TM* __restrict__ Ts,
                                                            const double* __restrict__ sdiag,
                                                            const double* __restrict__ b, double bscale,
                                                            double* __restrict__ dx, TM* wa, TM* wb,
                                                            double* partial, GridSync gs, double tol, int maxit,
                                                            PcgResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  const int stride = gridDim.x * blockDim.x;
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  double y[R], r[R], p[R], sv[R], z[R], w[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    y[u] = p[u] = sv[u] = z[u] = w[u] = 0.0;
    r[u] = 0.0;
    if (K < F.N) {
      r[u] = sdiag[K] * bscale * b[K];
      wa[K] = (TM)r[u];   // the first product is A r
    }
  }
  if (!grid_barrier(g)) return;
  double a4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    if (K < F.N) {
      w[u] = (double)sell_apply<TM>(F, Ts, wa, K);
      wb[K] = (TM)w[u];
      a4[0] = fma(r[u], r[u], a4[0]);
      a4[1] = fma(w[u], r[u], a4[1]);
    }
  }
  if (!grid_sum_x<2, 2>(g, a4, [&](double* o) {
        o[2] = 0.0;
        o[3] = o[1] != 0.0 ? o[0] / o[1] : 0.0;
      }))
    return;
  double gamma = a4[0], beta = a4[2], alpha = a4[3];
  const double rr0 = gamma;
  const double tol2 = tol * tol * rr0;
  TM* wc = wb;   // published w of the current iteration
  TM* wn = wa;   // next w
  int it = 0;
  while (rr0 > 0.0 && gamma > tol2 && it < maxit) {
    if (!(alpha != 0.0)) break;
    double n4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int K = k0 + u * stride;
      if (K < F.N) {
        const double nK = (double)sell_apply<TM>(F, Ts, wc, K);
        z[u] = nK + beta * z[u];
        sv[u] = w[u] + beta * sv[u];
        p[u] = r[u] + beta * p[u];
        y[u] += alpha * p[u];
        r[u] = r[u] - alpha * sv[u];
        w[u] = w[u] - alpha * z[u];
        wn[K] = (TM)w[u];
        n4[0] = fma(r[u], r[u], n4[0]);
        n4[1] = fma(w[u], r[u], n4[1]);
      }
    }
    if (!grid_sum_x<2, 2>(g, n4, [&](double* o) {
          const double g = o[0], d = o[1];
          const double bn = gamma != 0.0 ? g / gamma : 0.0;
          const double den = d - bn * g / alpha;
          o[2] = bn;
          o[3] = den != 0.0 ? g / den : 0.0;
        }))
      return;
    gamma = n4[0];
    beta = n4[2];
    alpha = n4[3];
    TM* t = wc;
    wc = wn;
    wn = t;
    ++it;
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    if (K < F.N) dx[K] = sdiag[K] * y[u];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = gamma;
  }
}

// (H v)_l for the lambdas of a warp-uniform group loop: a group of gsz lanes per lambda reads the two H rows of
// lambda_l (one per interface slot k, scaled by kappa of the slot's cell) with stride gsz and adds up by shuffles;
// v(lambda_j) is gathered through L2. Every lane returns the group sum.
template <class T>
__device__ __forceinline__ T hyb_row_product(const LevelDev& L, const T* __restrict__ Hc, const double* kapc,
                                             const T* v, int l, int g, int gsz, bool act) {
  T h = (T)0;
  if (act) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int k = side == 0 ? L.lam_y0[l] : L.lam_y1[l];
      const int c = L.if_cell[k];
      const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
      const T* Hk = Hc + L.hc_off[c] + (size_t)(k - k0) * ni;
      const int* lk = L.if_lam + k0;
      T y = 0;
      for (int j = g; j < ni; j += gsz) y += Hk[j] * __ldcg(&v[lk[j]]);
      h += (T)__ldcg(&kapc[c]) * y;
    }
  }
  for (int off = gsz >> 1; off > 0; off >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
  return h;
}

// Pipelined (Ghysels-Vanroose) Jacobi-preconditioned CG on H lambda = xi, one grid synchronisation per iteration.
// On entry lam = 0, r = xi, u = M r (M = diag(H)^-1) and rr0 = (r, r). State per lambda: lam, r, u, w = H u,
// z = H q, q = M s, s = H p, p; the vector m = M w, which the product n = H m gathers, is published
// double-buffered. Per iteration: n = H m; z = n + beta z; q = m + beta q; s = w + beta s; p = u + beta p;
// lam += alpha p; r -= alpha s; u -= alpha q; w -= alpha z; then gamma = (r, u), delta = (w, u), (r, r) in one
// reduction, from which the last step derives the next beta and alpha.
// (H v)_l from the assembled SELL form (one thread per lambda, the 32 lambdas of a slice read their entries
// coalesced); the entries, then the gathered v, are loaded eight at a time before the products. hsv was written
// earlier in the launch, so it is read through L2.
template <class T>
__device__ __forceinline__ T sell_h_product(const LevelDev& L, const T* hsv, const T* v, int l, bool act) {
  T h = (T)0;
  if (act) {
    const int w = L.hs_w[l >> 5];
    const int e0 = L.hs_off[l >> 5] + (l & 31);
    for (int j0 = 0; j0 < w; j0 += 8) {
      T hv[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + 32 * (j0 + u);
        const bool in = j0 + u < w;
        hv[u] = in ? __ldcg(&hsv[e]) : (T)0;
        xv[u] = in ? __ldcg(&v[L.hs_col[e]]) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) h = fma(hv[u], xv[u], h);
    }
  }
  return h;
}

// H v of lambda l in the memory-resident loop: SELL form if assembled (gsz = 1), else the per-cell blocks.
template <class T>
__device__ __forceinline__ T h_product(const LevelDev& L, const T* __restrict__ Hc, const T* hsv, const double* kapc,
                                       const T* v, int l, int gi, int gsz, bool act) {
  if (hsv) return sell_h_product<T>(L, hsv, v, l, act);
  return hyb_row_product<T>(L, Hc, kapc, v, l, gi, gsz, act);
}

template <class T>
__device__ bool hyb_pipe_loop(const LevelDev& L, const T* __restrict__ Hc, const T* hsv, const double* kapc, T* lam,
                              T* lr, T* lu, T* pp, T* lq, T* ldinv, const HybPipeBufs<T>& P, Grid& g, int gsz,
                              double tol2, double rr0, int maxit, int& it_out, double& rr_out) {
  const long total = (long)L.nlam * gsz;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  // w = H u, m = M w, and the first reduction
  double d3[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  {
    T a0 = (T)0, a1 = (T)0, a2 = (T)0;
    for (long tb = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); tb < total; tb += stride) {
      const long t = tb + lane;
      const bool act = t < total;
      const int l = act ? (int)(t / gsz) : 0;
      const int gi = lane & (gsz - 1);
      const T w = h_product<T>(L, Hc, hsv, kapc, lu, l, gi, gsz, act);
      if (act && gi == 0) {
        const T r = lr[l], u = lu[l];
        P.w[l] = w;
        P.ma[l] = ldinv[l] * w;
        P.z[l] = (T)0;
        P.s[l] = (T)0;
        lq[l] = (T)0;
        pp[l] = (T)0;
        a0 = fma(r, u, a0);
        a1 = fma(w, u, a1);
        a2 = fma(r, r, a2);
      }
    }
    d3[0] = (double)a0;
    d3[1] = (double)a1;
    d3[2] = (double)a2;
  }
  if (!grid_sum_x<3, 2>(g, d3, [&](double* o) {
        o[3] = 0.0;
        o[4] = o[1] != 0.0 ? o[0] / o[1] : 0.0;
      }))
    return false;
  double gamma = d3[0], rr = d3[2], beta = d3[3], alpha = d3[4];
  T* mc = P.ma;   // published m of the current iteration
  T* mn = P.mb;
  int it = 0;
  while (rr0 > 0.0 && rr > tol2 && it < maxit) {
    if (!(alpha != 0.0)) break;
    const T a = (T)alpha, b = (T)beta;
    T a0 = (T)0, a1 = (T)0, a2 = (T)0;
    for (long tb = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); tb < total; tb += stride) {
      const long t = tb + lane;
      const bool act = t < total;
      const int l = act ? (int)(t / gsz) : 0;
      const int gi = lane & (gsz - 1);
      const T n = h_product<T>(L, Hc, hsv, kapc, mc, l, gi, gsz, act);
      if (act && gi == 0) {
        const T w = P.w[l], m = ldinv[l] * w;
        const T z = n + b * P.z[l];
        const T q = m + b * lq[l];
        const T sv = w + b * P.s[l];
        const T p = lu[l] + b * pp[l];
        P.z[l] = z;
        lq[l] = q;
        P.s[l] = sv;
        pp[l] = p;
        lam[l] = lam[l] + a * p;
        const T r = lr[l] - a * sv;
        const T u = lu[l] - a * q;
        const T wn = w - a * z;
        lr[l] = r;
        lu[l] = u;
        P.w[l] = wn;
        mn[l] = ldinv[l] * wn;
        a0 = fma(r, u, a0);
        a1 = fma(wn, u, a1);
        a2 = fma(r, r, a2);
      }
    }
    double n5[5] = {(double)a0, (double)a1, (double)a2, 0.0, 0.0};
    if (!grid_sum_x<3, 2>(g, n5, [&](double* o) {
          const double gn = o[0], dn = o[1];
          const double bn = gamma != 0.0 ? gn / gamma : 0.0;
          const double den = dn - bn * gn / alpha;
          o[3] = bn;
          o[4] = den != 0.0 ? gn / den : 0.0;
        }))
      return false;
    gamma = n5[0];
    rr = n5[2];
    beta = n5[3];
    alpha = n5[4];
    T* tmp = mc;
    mc = mn;
    mn = tmp;
    ++it;
  }
  it_out = it;
  rr_out = rr;
  return true;
}

// Register-resident form of hyb_pipe_loop for levels whose lambdas fit in one pass of the grid (nlam * gsz <=
// threads): the group of gsz lanes that owns lambda l keeps it for the whole solve. Its leader keeps the CG state of
// l (w, z, s, p, q, u, r, lambda and the Jacobi weight) in registers, and every lane keeps the descriptors of its
// share of the two H rows of l (row offset, lambda-index offset, length, kappa of the slot's cell: all fixed during
// the solve), so an iteration's dependent loads are only the lane's H entries and lambda indices (independent of
// each other) and the gathered m values. m = M w is the one vector published per iteration (double-buffered);
// lambda is stored too, so that the recovery after the last reduction's barrier reads the final values.
template <class T>
__device__ bool hyb_pipe_loop_reg(const LevelDev& L, const T* __restrict__ Hc, const double* kapc, T* lam,
                                  const T* lr, const T* lu, const T* ldinv, const HybPipeBufs<T>& P, Grid& g,
                                  int gsz, double tol2, double rr0, int maxit, int& it_out, double& rr_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = t / gsz;
  const int gi = t & (gsz - 1);
  const bool act = l < L.nlam;
  const bool lead = act && gi == 0;
  int hb0 = 0, hb1 = 0, lb0 = 0, lb1 = 0, n0 = 0, n1 = 0;
  T kp0 = (T)0, kp1 = (T)0;
  if (act) {
    const int ka = L.lam_y0[l], kb = L.lam_y1[l];
    const int ca = L.if_cell[ka], cb = L.if_cell[kb];
    const int a0 = L.if_off[ca], b0 = L.if_off[cb];
    n0 = L.if_off[ca + 1] - a0;
    n1 = L.if_off[cb + 1] - b0;
    hb0 = L.hc_off[ca] + (ka - a0) * n0;
    hb1 = L.hc_off[cb] + (kb - b0) * n1;
    lb0 = a0;
    lb1 = b0;
    kp0 = (T)__ldcg(&kapc[ca]);
    kp1 = (T)__ldcg(&kapc[cb]);
  }
  // the group's share of (H v)_l, summed over the group by shuffles (every lane of the warp takes part)
  auto rowprod = [&](const T* v) -> T {
    T y0 = (T)0, y1 = (T)0;
    for (int j = gi; j < n0; j += gsz) y0 += Hc[hb0 + j] * __ldcg(&v[L.if_lam[lb0 + j]]);
    for (int j = gi; j < n1; j += gsz) y1 += Hc[hb1 + j] * __ldcg(&v[L.if_lam[lb1 + j]]);
    T h = kp0 * y0 + kp1 * y1;
    for (int off = gsz >> 1; off > 0; off >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
    return h;
  };
  T r = (T)0, u = (T)0, di = (T)0, lm = (T)0;
  if (lead) {
    r = __ldcg(&lr[l]);
    u = __ldcg(&lu[l]);
    di = __ldcg(&ldinv[l]);
  }
  T w = rowprod(lu);
  T z = (T)0, s = (T)0, q = (T)0, p = (T)0;
  double d3[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (lead) {
    P.ma[l] = di * w;
    d3[0] = (double)(r * u);
    d3[1] = (double)(w * u);
    d3[2] = (double)(r * r);
  }
  if (!grid_sum_x<3, 2>(g, d3, [&](double* o) {
        o[3] = 0.0;
        o[4] = o[1] != 0.0 ? o[0] / o[1] : 0.0;
      }))
    return false;
  double gamma = d3[0], rr = d3[2], beta = d3[3], alpha = d3[4];
  T* mc = P.ma;
  T* mn = P.mb;
  int it = 0;
  while (rr0 > 0.0 && rr > tol2 && it < maxit) {
    if (!(alpha != 0.0)) break;
    const T a = (T)alpha, b = (T)beta;
    const T n = rowprod(mc);
    double n5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (lead) {
      const T m = di * w;
      z = n + b * z;
      q = m + b * q;
      s = w + b * s;
      p = u + b * p;
      lm = lm + a * p;
      r = r - a * s;
      u = u - a * q;
      w = w - a * z;
      mn[l] = di * w;
      lam[l] = lm;
      n5[0] = (double)(r * u);
      n5[1] = (double)(w * u);
      n5[2] = (double)(r * r);
    }
    if (!grid_sum_x<3, 2>(g, n5, [&](double* o) {
          const double gn = o[0], dn = o[1];
          const double bn = gamma != 0.0 ? gn / gamma : 0.0;
          const double den = dn - bn * gn / alpha;
          o[3] = bn;
          o[4] = den != 0.0 ? gn / den : 0.0;
        }))
      return false;
    gamma = n5[0];
    rr = n5[2];
    beta = n5[3];
    alpha = n5[4];
    T* tmp = mc;
    mc = mn;
    mn = tmp;
    ++it;
  }
  it_out = it;
  rr_out = rr;
  return true;
}

// FP32 pipelined CG with residual replacement. The recurrences of the pipelined CG (kp_fine_cg_reg) run in FP32
// here, vectors and scaled matrix alike, a thread's cells in registers; in FP32 they drift away from the true
// residual on the six-decade channelized field (the iteration count grew fivefold), so every `replace` iterations
// the residual and the auxiliary vectors are recomputed from their definitions -- r = b - A y, s = A p, then
// w = A r and z = A s (residual replacement, Cools and Vanroose) -- which costs four matrix products and two extra
// synchronisations and keeps the iteration on the track of the FP64 one. Per-thread partial sums in FP32, block and
// grid sums in FP64; the stopping test and the step lengths are those of kp_fine_cg_reg.
template <int R>
__global__ void __launch_bounds__(kPThreads) kp_fine_cg_rr32(FineDev F, const float* __restrict__ Ts,
                                                             const double* __restrict__ sdiag,
                                                             const double* __restrict__ b, double bscale,
                                                             double* __restrict__ dx, float* wa, float* wb,
                                                             float* ypub, float* ppub, float* rpub, float* spub,
                                                             double* partial, GridSync gs, double tol, int maxit,
                                                             int replace, PcgResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  const int stride = gridDim.x * blockDim.x;
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  float y[R], r[R], p[R], sv[R], z[R], w[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    y[u] = p[u] = sv[u] = z[u] = w[u] = r[u] = 0.0f;
    if (K < F.N) {
      r[u] = (float)(sdiag[K] * bscale * b[K]);
      wa[K] = r[u];   // the first product is A r
    }
  }
  if (!grid_barrier(g)) return;
  float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    if (K < F.N) {
      w[u] = sell_apply<float>(F, Ts, wa, K);
      wb[K] = w[u];
      t0 = fmaf(r[u], r[u], t0);
      t1 = fmaf(w[u], r[u], t1);
    }
  }
  double a4[4] = {(double)t0, (double)t1, 0.0, 0.0};
  if (!grid_sum_x<2, 2>(g, a4, [&](double* o) {
        o[2] = 0.0;
        o[3] = o[1] != 0.0 ? o[0] / o[1] : 0.0;
      }))
    return;
  double gamma = a4[0], beta = a4[2], alpha = a4[3];
  const double rr0 = gamma;
  const double tol2 = tol * tol * rr0;
  float* wc = wb;   // published w of the current iteration
  float* wn = wa;   // next w
  int it = 0;
  while (rr0 > 0.0 && gamma > tol2 && it < maxit) {
    if (!(alpha != 0.0)) break;
    const float af = (float)alpha, bf = (float)beta;
    float n0 = 0.0f, n1 = 0.0f;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int K = k0 + u * stride;
      if (K < F.N) {
        const float nK = sell_apply<float>(F, Ts, wc, K);
        z[u] = nK + bf * z[u];
        sv[u] = w[u] + bf * sv[u];
        p[u] = r[u] + bf * p[u];
        y[u] += af * p[u];
        r[u] = r[u] - af * sv[u];
        w[u] = w[u] - af * z[u];
        wn[K] = w[u];
        n0 = fmaf(r[u], r[u], n0);
        n1 = fmaf(w[u], r[u], n1);
      }
    }
    if (replace > 0 && (it + 1) % replace == 0) {
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int K = k0 + u * stride;
        if (K < F.N) {
          ypub[K] = y[u];
          ppub[K] = p[u];
        }
      }
      if (!grid_barrier(g)) return;
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int K = k0 + u * stride;
        if (K < F.N) {
          r[u] = (float)(sdiag[K] * bscale * b[K]) - sell_apply<float>(F, Ts, ypub, K);
          sv[u] = sell_apply<float>(F, Ts, ppub, K);
          rpub[K] = r[u];
          spub[K] = sv[u];
        }
      }
      if (!grid_barrier(g)) return;
      n0 = n1 = 0.0f;
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int K = k0 + u * stride;
        if (K < F.N) {
          w[u] = sell_apply<float>(F, Ts, rpub, K);
          z[u] = sell_apply<float>(F, Ts, spub, K);
          wn[K] = w[u];
          n0 = fmaf(r[u], r[u], n0);
          n1 = fmaf(w[u], r[u], n1);
        }
      }
    }
    double n4[4] = {(double)n0, (double)n1, 0.0, 0.0};
    if (!grid_sum_x<2, 2>(g, n4, [&](double* o) {
          const double g = o[0], d = o[1];
          const double bn = gamma != 0.0 ? g / gamma : 0.0;
          const double den = d - bn * g / alpha;
          o[2] = bn;
          o[3] = den != 0.0 ? g / den : 0.0;
        }))
      return;
    gamma = n4[0];
    beta = n4[2];
    alpha = n4[3];
    float* t = wc;
    wc = wn;
    wn = t;
    ++it;
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int K = k0 + u * stride;
    if (K < F.N) dx[K] = sdiag[K] * (double)y[u];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = gamma;
  }
}

// ---- fine level: Newton update J dx = bscale * b with the exact Jacobian ---------------------------------------
// Row K of the scaled Jacobian applied to v: jd_K v_K + sum_e Js_e v_L(e) (SELL-32 layout; padding entries are 0).
__device__ __forceinline__ double jac_row(const FineDev& F, const double* __restrict__ Js, double jdK, const double* v,
                                          int K) {
  const int s = K >> 5, lane = K & 31;
  double acc = jdK * __ldcg(&v[K]);
  const int w = F.sell_w[s];
  int e = F.sell_off[s] + lane;
  int j = 0;
  if (w <= 8) {
    int Ls[8];
    double Jv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < w) {
        Ls[u] = F.nbr[e + 32 * u];
        Jv[u] = Js[e + 32 * u];
      }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < w) acc = fma(Jv[u], __ldcg(&v[Ls[u]]), acc);
    j = w;
  }
  for (e += 32 * j; j < w; ++j, e += 32) acc = fma(Js[e], __ldcg(&v[F.nbr[e]]), acc);
  return acc;
}

// BiCGStab (van der Vorst) in FP64 on the symmetrically scaled Newton system (S J S) y = S bscale b, dx = S y, with
// S = D^1/2 and D = 1 / max(J_KK, d_K / 2) the weights of the nonlinear Jacobi smoother (d_K the frozen-coefficient
// diagonal); jd = J_KK D_K and Js = S_K J_KL S_L are formed before the launch. The Jacobian is not symmetric, so CG
// does not apply; BiCGStab's short recurrences keep the whole solve in one persistent launch with a fixed amount of
// memory. One iteration: v = A p and (rh, v) give alpha; s = r - alpha v is published; t = A s, (t, s) and (t, t)
// give omega; y += alpha p + omega s, r = s - omega t, (rh, r) and (r, r) give rho and beta; p = r + beta (p - omega
// v) is published: three reductions and two plain barriers. The stopping test is ||r|| <= tol ||r_0|| on the scaled
// residual, as for the CG; a breakdown (alpha, omega or rho zero) ends the solve with the current y.
__global__ void __launch_bounds__(kPThreads) kp_fine_bicgstab(FineDev F, const double* __restrict__ Js,
                                                              const double* __restrict__ jd,
                                                              const double* __restrict__ sS,
                                                              const double* __restrict__ b, double bscale,
                                                              double* __restrict__ dx, double* __restrict__ y,
                                                              double* __restrict__ r, double* __restrict__ rh,
                                                              double* p, double* __restrict__ v, double* s,
                                                              double* __restrict__ t, double* partial, GridSync gs,
                                                              double tol, int maxit, PcgResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  double a1[1] = {0.0};
  GSTRIDE(i, F.N) {
    const double ri = sS[i] * bscale * b[i];
    y[i] = 0.0;
    r[i] = ri;
    rh[i] = ri;
    p[i] = ri;
    a1[0] = fma(ri, ri, a1[0]);
  }
  if (!grid_sum<1>(g, a1)) return;   // its barrier also publishes p
  const double rr0 = a1[0];
  double rr = rr0, rho = rr0;
  const double tol2 = tol * tol * rr0;
  int it = 0;
  while (rr0 > 0.0 && rr > tol2 && it < maxit) {
    double a2[2] = {0.0, 0.0};
    GSTRIDE(K, F.N) {
      const double vK = jac_row(F, Js, jd[K], p, K);
      v[K] = vK;
      a2[0] = fma(rh[K], vK, a2[0]);
    }
    if (!grid_sum_x<1, 1>(g, a2, [&](double* o) { o[1] = o[0] != 0.0 ? rho / o[0] : 0.0; })) return;
    const double alpha = a2[1];
    if (!(alpha != 0.0)) break;
    GSTRIDE(K, F.N) s[K] = r[K] - alpha * v[K];
    if (!grid_barrier(g)) return;
    double a3[3] = {0.0, 0.0, 0.0};
    GSTRIDE(K, F.N) {
      const double tK = jac_row(F, Js, jd[K], s, K);
      const double sK = s[K];
      t[K] = tK;
      a3[0] = fma(tK, sK, a3[0]);
      a3[1] = fma(tK, tK, a3[1]);
    }
    if (!grid_sum_x<2, 1>(g, a3, [&](double* o) { o[2] = o[1] != 0.0 ? o[0] / o[1] : 0.0; })) return;
    const double omega = a3[2];
    double a4[3] = {0.0, 0.0, 0.0};
    GSTRIDE(K, F.N) {
      const double sK = s[K];
      y[K] += alpha * p[K] + omega * sK;
      const double rK = sK - omega * t[K];
      r[K] = rK;
      a4[0] = fma(rh[K], rK, a4[0]);
      a4[1] = fma(rK, rK, a4[1]);
    }
    if (!grid_sum_x<2, 1>(g, a4, [&](double* o) {
          o[2] = rho != 0.0 && omega != 0.0 ? (o[0] / rho) * (alpha / omega) : 0.0;
        }))
      return;
    ++it;
    rr = a4[1];
    const double beta = a4[2];
    const bool stop = !(omega != 0.0) || !(a4[0] != 0.0);
    rho = a4[0];
    if (stop) break;
    GSTRIDE(K, F.N) p[K] = r[K] + beta * (p[K] - omega * v[K]);
    if (!grid_barrier(g)) return;
  }
  GSTRIDE(i, F.N) dx[i] = sS[i] * y[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = rr;
  }
}

// ---- coarse level: hybridized saddle solve (rhs, Jacobi diagonal, CG on H lambda = xi, local recovery) ------
// The solve of one frozen-coefficient coarse saddle as a device function of a persistent grid (g.sm: kSmDoubles of
// shared memory). kapc, bs and bp may have been written earlier in the same launch, so they are read through L2.
// Returns false if a grid barrier gave up; `iters` and `rr_out` receive the CG iterations and final (r, r).
template <class T>
__device__ bool hyb_solve_dev(const LevelDev& L, const T* __restrict__ Hc, const T* __restrict__ Sinv,
                              const double* kapc, const double* bs, const double* bp, T* ylam, T* ydiag, T* lam,
                              T* lr, T* lz, T* pa, T* pb, T* lq, T* ldinv, double* dsig, double* dp, Grid& g,
                              double tol, int maxit, int gsz, int& iters, double& rr0_out, double& rr_out,
                              const HybPipeBufs<T>* pipe = nullptr, int gsz_reg = 0, T* hsv = nullptr) {
  // phase 0: per interface slot k of cell c, u_k = kappa A[k,:] bhat + B[k,:] b_p (signed) and kappa Hc[k,k]
  GSTRIDE(k, L.nif) {
    const int c = L.if_cell[k];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const double kp = __ldcg(&kapc[c]);
    const int u = L.if_slot[k];
    const T* Su = Sinv + L.sad_off[c] + (size_t)u * n;
    T a1 = 0, a2_ = 0;
    for (int t = 0; t < nl; ++t)
      if (L.own0[lo + t]) a1 += Su[t] * (T)__ldcg(&bs[L.loc[lo + t]]);
    for (int q = 0; q < mc; ++q) a2_ += Su[nl + q] * (T)__ldcg(&bp[po + q]);
    ylam[k] = (T)L.if_sign[k] * ((T)kp * a1 + a2_);
    const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
    ydiag[k] = (T)kp * Hc[L.hc_off[c] + (k - k0) * ni + (k - k0)];
  }
  if (hsv) {   // the SELL form of H at this kappa (padding entries have no contribution: 0)
    GSTRIDE(l, L.nlam) {
      const T k0 = (T)__ldcg(&kapc[L.lam_c0[l]]), k1 = (T)__ldcg(&kapc[L.lam_c1[l]]);
      const int w = L.hs_w[l >> 5];
      int e = L.hs_off[l >> 5] + (l & 31);
      for (int j = 0; j < w; ++j, e += 32) {
        const int a = L.hs_i0[e], b = L.hs_i1[e];
        hsv[e] = (a >= 0 ? k0 * Hc[a] : (T)0) + (b >= 0 ? k1 * Hc[b] : (T)0);
      }
    }
  }
  if (!grid_barrier(g)) return false;
  T u0 = (T)0, u1 = (T)0;   // per-thread partial sums in T, block and grid sums in FP64
  GSTRIDE(l, L.nlam) {
    const T xi = __ldcg(&ylam[L.lam_y0[l]]) + __ldcg(&ylam[L.lam_y1[l]]);
    const T di = (T)1 / (__ldcg(&ydiag[L.lam_y0[l]]) + __ldcg(&ydiag[L.lam_y1[l]]));
    ldinv[l] = di;
    lam[l] = (T)0;
    lr[l] = xi;
    const T zi = xi * di;
    lz[l] = zi;
    u0 = fma(xi, zi, u0);
    u1 = fma(xi, xi, u1);
  }
  double a2[2] = {(double)u0, (double)u1};
  if (!grid_sum<2>(g, a2)) return false;
  double rz = a2[0];
  const double rr0 = a2[1];
  double rr = rr0;
  const double tol2 = tol * tol * rr0;
  T beta = (T)0;
  T* pp = pa;       // search direction p
  int it = 0;
  if (pipe && gsz_reg > 0) {
    if (!hyb_pipe_loop_reg<T>(L, Hc, kapc, lam, lr, lz, ldinv, *pipe, g, gsz_reg, tol2, rr0, maxit, it, rr))
      return false;
  } else if (pipe) {
    if (!hyb_pipe_loop<T>(L, Hc, hsv, kapc, lam, lr, lz, pp, lq, ldinv, *pipe, g, hsv ? 1 : gsz, tol2, rr0, maxit,
                          it, rr))
      return false;
  }
  while (!pipe && rr0 > 0.0 && rr > tol2 && it < maxit) {
    // (H z)_l = sum over the two interface slots k of lambda_l of kappa_c Hc[k, :] z(lambda of c's slots): a group
    // of gsz lanes per lambda (gsz a power of two <= 32, chosen so that small coarse levels still occupy every SM)
    // reads both rows with stride gsz and adds up by shuffles, so H z needs no intermediate buffer and no extra
    // barrier; H p then follows by recurrence. z was published by the previous reduction's barrier.
    T upq = (T)0;
    {
      const long total = (long)L.nlam * gsz;
      const int lane = threadIdx.x & 31;
      const long stride = (long)gridDim.x * blockDim.x;
      for (long tb = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); tb < total; tb += stride) {
        const long t = tb + lane;   // warp-uniform loop: every lane takes part in the shuffles
        const bool act = t < total;
        const int l = act ? (int)(t / gsz) : 0;
        const int g = lane & (gsz - 1);
        T hz = (T)0;
        if (act) {
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const int k = side == 0 ? L.lam_y0[l] : L.lam_y1[l];
            const int c = L.if_cell[k];
            const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
            const T* Hk = Hc + L.hc_off[c] + (size_t)(k - k0) * ni;
            const int* lk = L.if_lam + k0;
            T y = 0;
            for (int j = g; j < ni; j += gsz) y += Hk[j] * __ldcg(&lz[lk[j]]);
            hz += (T)__ldcg(&kapc[c]) * y;
          }
        }
        for (int off = gsz >> 1; off > 0; off >>= 1) hz += __shfl_xor_sync(0xffffffffu, hz, off);
        if (act && g == 0) {
          const T zl = lz[l];
          const T pl = it == 0 ? zl : zl + beta * pp[l];
          const T ql = it == 0 ? hz : hz + beta * lq[l];
          pp[l] = pl;
          lq[l] = ql;
          upq = fma(pl, ql, upq);
        }
      }
    }
    double a1[2] = {(double)upq, 0.0};
    if (!grid_sum_x<1, 1>(g, a1, [&](double* o) { o[1] = o[0] != 0.0 ? rz / o[0] : 0.0; }))
      return false;
    const double alpha_d = a1[1];
    const T alpha = (T)alpha_d;
    u0 = u1 = (T)0;
    GSTRIDE(l, L.nlam) {
      lam[l] = alpha * pp[l] + lam[l];
      const T ri = lr[l] - alpha * lq[l];
      const T zi = ri * ldinv[l];
      lr[l] = ri;
      lz[l] = zi;
      u0 = fma(ri, zi, u0);
      u1 = fma(ri, ri, u1);
    }
    double a3[3] = {(double)u0, (double)u1, 0.0};
    if (!grid_sum_x<2, 1>(g, a3, [&](double* o) { o[2] = rz != 0.0 ? o[0] / rz : 0.0; }))
      return false;
    beta = (T)a3[2];
    rz = a3[0];
    rr = a3[1];
    ++it;
    if (!(alpha_d != 0.0)) break;
  }
  // recovery: sigma^c = kappa A w + B b_p, p_c = B^T w + C b_p / kappa with w = bhat - C^T lambda; one thread per
  // owned local flux slot, then one per pressure unknown
  GSTRIDE(y, L.nyl) {
    if (!L.own0[y]) continue;
    const int c = L.slot_cell[y];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const int u = y - lo;
    const T* Su = Sinv + L.sad_off[c] + (size_t)u * n;
    T a1 = 0, a2_ = 0;
    for (int t = 0; t < nl; ++t)
      if (L.own0[lo + t]) a1 += Su[t] * (T)__ldcg(&bs[L.loc[lo + t]]);
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k)
      a1 -= Su[L.if_slot[k]] * (T)L.if_sign[k] * __ldcg(&lam[L.if_lam[k]]);
    for (int q = 0; q < mc; ++q) a2_ += Su[nl + q] * (T)__ldcg(&bp[po + q]);
    dsig[L.loc[y]] = (double)((T)__ldcg(&kapc[c]) * a1 + a2_);
  }
  GSTRIDE(i, L.np) {
    const int c = L.p_cell[i];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const T* Sr = Sinv + L.sad_off[c] + (size_t)(nl + i - po) * n;
    T a1 = 0, a2_ = 0;
    for (int t = 0; t < nl; ++t)
      if (L.own0[lo + t]) a1 += Sr[t] * (T)__ldcg(&bs[L.loc[lo + t]]);
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k)
      a1 -= Sr[L.if_slot[k]] * (T)L.if_sign[k] * __ldcg(&lam[L.if_lam[k]]);
    for (int q = 0; q < mc; ++q) a2_ += Sr[nl + q] * (T)__ldcg(&bp[po + q]);
    dp[i] = (double)a1 + (double)a2_ / __ldcg(&kapc[c]);
  }
  iters = it;
  rr0_out = rr0;
  rr_out = rr;
  return true;
}


// ---- fused coarse Picard step -------------------------------------------------------------------------------
// The coarse operator (Prop. 1, eq. structure) is linear in [sigma; p] once kappa is fixed: with kappa_c =
// kappa((Pi~ p)_c), A(x)_sigma,i = sum over the (one or two) owner slots y of flux unknown i of
// (M_c sigma_c)_u / kappa_c + (D_c^T p_c)_u and A(x)_p,i = (D_c sigma_c)_i. Algorithm 1 evaluates A at x + s dx for
// several s; the linear parts of x and of dx (LinParts) are computed once, and each trial is then one pass over the
// flux and pressure unknowns -- (ms_x + s ms_dx) / kappa(pb_x + s pb_dx) + ds_x + s ds_dx -- and one reduction,
// instead of a whole operator evaluation with two synchronisations. On this part the FP64 products of an
// evaluation and its synchronisations are what a coarse step costs, not its bytes.

// Linear parts of v (read through L2: v may have been written earlier in the launch). With shift != 0 the parts
// `acc` first take acc += shift * out (the previous step's accepted trial; the same lane owns both entries).
__device__ void lin_parts_pass(const LevelDev& L, const double* v, LinParts out, LinParts acc, double shift) {
  const double* vs = v;
  const double* vp = v + L.nflux;
  GSTRIDE(y, L.nyl) {
    const int c = L.slot_cell[y];
    const int lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, mc = L.m[c], po = L.p_off[c];
    const int u = y - lo;
    const double* Mu = L.Mloc + L.mat_off[c] + (size_t)u * nl;
    const double* D = L.Dloc + L.dmat_off[c];
    double m = 0.0, d = 0.0;
    for (int k = 0; k < nl; ++k) m = fma(Mu[k], __ldcg(&vs[L.loc[lo + k]]), m);
    for (int q = 0; q < mc; ++q) d = fma(D[q * nl + u], __ldcg(&vp[po + q]), d);
    if (shift != 0.0) {
      acc.ms[y] = fma(shift, out.ms[y], acc.ms[y]);
      acc.ds[y] = fma(shift, out.ds[y], acc.ds[y]);
    }
    out.ms[y] = m;
    out.ds[y] = d;
  }
  GSTRIDE(i, L.np) {
    const int c = L.p_cell[i];
    const int lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c];
    const double* Dr = L.Dloc + L.dmat_off[c] + (size_t)(i - po) * nl;
    double d = 0.0;
    for (int k = 0; k < nl; ++k) d = fma(Dr[k], __ldcg(&vs[L.loc[lo + k]]), d);
    if (shift != 0.0) acc.dr[i] = fma(shift, out.dr[i], acc.dr[i]);
    out.dr[i] = d;
  }
  GSTRIDE(c, L.nc) {
    const int po = L.p_off[c];
    double pb = 0.0;
    for (int q = 0; q < L.m[c]; ++q) pb = fma(L.w[po + q], __ldcg(&vp[po + q]), pb);
    if (shift != 0.0) acc.pb[c] = fma(shift, out.pb[c], acc.pb[c]);
    out.pb[c] = pb;
  }
}

// A(x + s dx) - b from the linear parts (dir is not read when s == 0), for flux unknown i / pressure unknown i.
__device__ __forceinline__ double trial_flux_row(const LevelDev& L, const LinParts& bx, const LinParts& dx, double s,
                                                 const double* b, int kind, double a, int i) {
  double v = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int y = side == 0 ? L.f_y0[i] : L.f_y1[i];
    if (y < 0) continue;
    const int c = L.slot_cell[y];
    double pb = __ldcg(&bx.pb[c]), m = __ldcg(&bx.ms[y]), d = __ldcg(&bx.ds[y]);
    if (s != 0.0) {
      pb = fma(s, __ldcg(&dx.pb[c]), pb);
      m = fma(s, __ldcg(&dx.ms[y]), m);
      d = fma(s, __ldcg(&dx.ds[y]), d);
    }
    v += fma(m, inv_kappa_of(pb, kind, a), d);
  }
  return v - __ldcg(&b[i]);
}
__device__ __forceinline__ double trial_p_row(const LevelDev& L, const LinParts& bx, const LinParts& dx, double s,
                                              const double* b, int i) {
  double d = __ldcg(&bx.dr[i]);
  if (s != 0.0) d = fma(s, __ldcg(&dx.dr[i]), d);
  return d - __ldcg(&b[L.nflux + i]);
}

// ||A(x + s dx) - b|| (one pass, one reduction).
__device__ bool trial_norm(const LevelDev& L, const LinParts& bx, const LinParts& dx, double s, const double* b,
                           int kind, double a, Grid& g, double& rn) {
  double acc = 0.0;
  GSTRIDE(i, L.nflux) {
    const double v = trial_flux_row(L, bx, dx, s, b, kind, a, i);
    acc = fma(v, v, acc);
  }
  GSTRIDE(i, L.np) {
    const double v = trial_p_row(L, bx, dx, s, b, i);
    acc = fma(v, v, acc);
  }
  double s1[1] = {acc};
  if (!grid_sum<1>(g, s1)) return false;
  rn = sqrt(s1[0]);
  return true;
}

// Makes x + s dx the iterate: r = A(x) - b, nb = -r and kappa per cell at the new point, x += s dx; returns this
// thread's share of ||r||^2 (the same sum as the trial's). The linear parts of x are left as they were (the next
// pass over the step's direction adds s times the old direction's).
template <class T>
__device__ double accept_pass(const LevelDev& L, const CoarseStepBufs<T>& B, double s, int kind, double a) {
  double acc = 0.0;
  GSTRIDE(i, L.nflux) {
    const double v = trial_flux_row(L, B.base, B.dir, s, B.b, kind, a, i);
    B.r[i] = v;
    B.nb[i] = -v;
    acc = fma(v, v, acc);
  }
  GSTRIDE(i, L.np) {
    const double v = trial_p_row(L, B.base, B.dir, s, B.b, i);
    B.r[L.nflux + i] = v;
    B.nb[L.nflux + i] = -v;
    acc = fma(v, v, acc);
  }
  GSTRIDE(c, L.nc) {
    double pb = __ldcg(&B.base.pb[c]);
    if (s != 0.0) pb = fma(s, __ldcg(&B.dir.pb[c]), pb);
    B.kapc[c] = kappa_of(pb, kind, a);
  }
  if (s != 0.0) {
    const int nx = L.nflux + L.np;
    GSTRIDE(i, nx) B.x[i] = fma(s, __ldcg(&B.dx[i]), B.x[i]);
  }
  return acc;
}

// Algorithm 1 from x (residual norm rn) along s0 dx, with trial norms from the linear parts. Returns the accepted
// scaling s * s0 in `step` (0: every trial was non-finite, x is kept; a non-finite trial counts as +infinity) and its
// residual norm in rn.
__device__ bool backtrack_lin(const LevelDev& L, const LinParts& bx, const LinParts& dx, const CoarseStepParams& P,
                              const double* b, double s0, double& rn, double& step, int& trials, Grid& g) {
  double s = 1.0, r_s = 0.0;
  if (!trial_norm(L, bx, dx, s * s0, b, P.kind, P.a, g, r_s)) return false;
  ++trials;
  if (!isfinite(r_s)) r_s = HUGE_VAL;
  int n = 0;
  while (r_s > rn && n < P.bt_nmax) {
    double r_half = 0.0;
    if (!trial_norm(L, bx, dx, 0.5 * s * s0, b, P.kind, P.a, g, r_half)) return false;
    ++trials;
    if (!isfinite(r_half)) r_half = HUGE_VAL;
    if (r_half > P.bt_theta * r_s) break;
    s *= 0.5;
    ++n;
    r_s = r_half;
  }
  if (r_s == HUGE_VAL) {
    step = 0.0;
    return true;
  }
  step = s * s0;
  rn = r_s;
  return true;
}

// One launch. On entry x (and, with backtrack_first, the correction in dx and ||A(x) - b|| in rn_in); on exit x, r,
// nb = -r and kappa per cell at the final x.
template <class T>
__global__ void __launch_bounds__(kPThreads, 1) kp_coarse_step(LevelDev L, const T* __restrict__ Hc,
                                                           const T* __restrict__ Sinv, CoarseStepBufs<T> B,
                                                           CoarseStepParams P, double* partial, GridSync gs,
                                                           int gsz, int gsz_reg, CoarseStepResult* res) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  int iters = 0, steps = 0, evals = 0, trials = 0, bad = 0;
  double rn = P.rn_in;
  double pending = 0.0;   // accepted step not yet added to the linear parts of x
  // linear parts of x (and of the given correction)
  lin_parts_pass(L, B.x, B.base, B.base, 0.0);
  ++evals;
  if (P.backtrack_first) {
    lin_parts_pass(L, B.dx, B.dir, B.dir, 0.0);
    ++evals;
  }
  if (!grid_barrier(g)) return;
  double step = 0.0;
  if (P.backtrack_first) {
    if (!backtrack_lin(L, B.base, B.dir, P, B.b, 1.0, rn, step, trials, g)) return;
  }
  const double acc = accept_pass<T>(L, B, step, P.kind, P.a);   // r, nb, kappa at the (new) x
  pending = step;
  if (!P.backtrack_first) {
    double s1[1] = {acc};
    if (!grid_sum<1>(g, s1)) return;
    rn = sqrt(s1[0]);
    if (!isfinite(rn)) bad = 1;
  } else if (!grid_barrier(g)) {
    return;
  }
  const double r0 = rn;
  for (int k = 0; k < P.nsteps && !bad; ++k) {
    if (P.coarsest && (rn <= P.tol_rel * r0 || rn <= P.tol_abs)) break;
    int it = 0;
    double rr0 = 0.0, rr = 0.0;
    if (!hyb_solve_dev<T>(L, Hc, Sinv, B.kapc, B.nb, B.nb + L.nflux, B.ylam, B.ydiag, B.lam, B.lr, B.lz, B.pa,
                          B.pb, B.lq, B.ldinv, B.dx, B.dx + L.nflux, g, P.lin_tol, P.maxit, gsz, it, rr0, rr,
                          B.pipe.w ? &B.pipe : nullptr, gsz_reg,
                          B.pipe.w && gsz_reg == 0 && L.hs_n > 0 ? B.hsv : nullptr))
      return;
    iters += it;
    if (!isfinite(rr)) {
      bad = 2;
      break;
    }
    if (!grid_barrier(g)) return;   // dx complete
    // linear parts of dx (after folding the previous accepted step into those of x), and the clamp on Pi~ dp
    lin_parts_pass(L, B.dx, B.dir, B.base, pending);
    ++evals;
    double s0 = 1.0;
    if (P.dp_clamp > 0.0) {
      double m = 0.0;
      GSTRIDE(c, L.nc) m = fmax(m, fabs(B.dir.pb[c]));   // written by this thread just above
      if (!grid_max(g, m)) return;
      if (m > P.dp_clamp) s0 = P.dp_clamp / m;
    } else if (!grid_barrier(g)) {
      return;
    }
    if (!backtrack_lin(L, B.base, B.dir, P, B.b, s0, rn, step, trials, g)) return;
    (void)accept_pass<T>(L, B, step, P.kind, P.a);
    pending = step;
    if (!grid_barrier(g)) return;   // r, nb, kappa and x complete
    ++steps;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->rn = rn;
    res->iters = iters;
    res->steps = steps;
    res->res_evals = evals;
    res->bad = bad;
    res->trials = trials;
  }
}

int coop_grid(const void* fn, int n_items, int sm_cap) {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPThreads, 0);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;                   // few, wide blocks: cheap barriers and partial sums
  const int use = sm_cap > 0 && sm_cap < sms ? sm_cap : sms;
  int maxb = use * per_sm;
  int need = (n_items + kPThreads - 1) / kPThreads;
  if (need < 1) need = 1;
  return need < maxb ? need : maxb;
}

}  // namespace

template <class T>
cudaError_t launch_fine_cg(cudaStream_t st, const FineDev& F, const T* Ts, const double* sdiag, const double* b,
                           double bscale, double* dx, T* y, T* r, T* pa, T* pb, T* q, double* partial, GridSync gs,
                           double tol, int maxit, PcgResult* res) {
  (void)pb;
  const void* fn = (const void*)kp_fine_cg<T>;
  int grid = coop_grid(fn, F.N, gs.sm_cap);
  void* args[] = {(void*)&F, (void*)&Ts, (void*)&sdiag, (void*)&b, (void*)&bscale, (void*)&dx, (void*)&y,
                  (void*)&r, (void*)&pa, (void*)&q, (void*)&partial, (void*)&gs, (void*)&tol,
                  (void*)&maxit, (void*)&res};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}
template <class T>
cudaError_t launch_fine_cg_pipe(cudaStream_t st, const FineDev& F, const T* Ts, const double* sdiag, const double* b,
                                double bscale, double* dx, T* y, T* r, T* wa, T* wb, T* z, T* sv, T* p,
                                double* partial, GridSync gs, double tol, int maxit, PcgResult* res) {
  const void* fn = (const void*)kp_fine_cg_pipe<T>;
  int grid = coop_grid(fn, F.N, gs.sm_cap);
  void* args[] = {(void*)&F, (void*)&Ts, (void*)&sdiag, (void*)&b, (void*)&bscale, (void*)&dx, (void*)&y,
                  (void*)&r, (void*)&wa, (void*)&wb, (void*)&z, (void*)&sv, (void*)&p, (void*)&partial, (void*)&gs,
                  (void*)&tol, (void*)&maxit, (void*)&res};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}
// FP32 pipelined CG with residual replacement if every thread holds at most 8 cells on the grid the launch gets;
// returns cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t launch_fine_cg_rr32(cudaStream_t st, const FineDev& F, const float* Ts, const double* sdiag,
                                const double* b, double bscale, double* dx, float* wa, float* wb, float* ypub,
                                float* ppub, float* rpub, float* spub, double* partial, GridSync gs, double tol,
                                int maxit, int replace, PcgResult* res) {
  const void* fns[4] = {(const void*)kp_fine_cg_rr32<1>, (const void*)kp_fine_cg_rr32<2>,
                        (const void*)kp_fine_cg_rr32<4>, (const void*)kp_fine_cg_rr32<8>};
  const int Rs[4] = {1, 2, 4, 8};
  for (int i = 0; i < 4; ++i) {
    const int grid = coop_grid(fns[i], F.N, gs.sm_cap);
    const long cap = (long)grid * kPThreads * Rs[i];
    if (cap < F.N) continue;
    void* args[] = {(void*)&F, (void*)&Ts, (void*)&sdiag, (void*)&b, (void*)&bscale, (void*)&dx, (void*)&wa,
                    (void*)&wb, (void*)&ypub, (void*)&ppub, (void*)&rpub, (void*)&spub, (void*)&partial,
                    (void*)&gs, (void*)&tol, (void*)&maxit, (void*)&replace, (void*)&res};
    return cudaLaunchCooperativeKernel(fns[i], dim3(grid), dim3(kPThreads), args, 0, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_fine_bicgstab(cudaStream_t st, const FineDev& F, const double* Js, const double* jd,
                                 const double* sS, const double* b, double bscale, double* dx, double* work,
                                 double* partial, GridSync gs, double tol, int maxit, PcgResult* res) {
  const void* fn = (const void*)kp_fine_bicgstab;
  const int grid = coop_grid(fn, F.N, gs.sm_cap);
  const size_t n = (size_t)F.N;
  double *y = work, *r = work + n, *rh = work + 2 * n, *p = work + 3 * n, *v = work + 4 * n, *s = work + 5 * n,
         *t = work + 6 * n;
  void* args[] = {(void*)&F, (void*)&Js, (void*)&jd, (void*)&sS, (void*)&b, (void*)&bscale, (void*)&dx,
                  (void*)&y, (void*)&r, (void*)&rh, (void*)&p, (void*)&v, (void*)&s, (void*)&t, (void*)&partial,
                  (void*)&gs, (void*)&tol, (void*)&maxit, (void*)&res};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}
// Register-resident pipelined CG if every thread holds at most 4 cells on the grid the launch gets; returns
// cudaErrorNotSupported (nothing launched) otherwise.
template <class TM>
cudaError_t launch_fine_cg_reg(cudaStream_t st, const FineDev& F, const TM* Ts, const double* sdiag, const double* b,
                               double bscale, double* dx, TM* wa, TM* wb, double* partial, GridSync gs, double tol,
                               int maxit, PcgResult* res) {
  const void* fns[3] = {(const void*)kp_fine_cg_reg<TM, 1>, (const void*)kp_fine_cg_reg<TM, 2>,
                        (const void*)kp_fine_cg_reg<TM, 4>};
  const int Rs[3] = {1, 2, 4};
  for (int i = 0; i < 3; ++i) {
    const int grid = coop_grid(fns[i], F.N, gs.sm_cap);
    const long cap = (long)grid * kPThreads * Rs[i];
    if (cap < F.N) continue;
    void* args[] = {(void*)&F, (void*)&Ts, (void*)&sdiag, (void*)&b, (void*)&bscale, (void*)&dx, (void*)&wa,
                    (void*)&wb, (void*)&partial, (void*)&gs, (void*)&tol, (void*)&maxit, (void*)&res};
    return cudaLaunchCooperativeKernel(fns[i], dim3(grid), dim3(kPThreads), args, 0, st);
  }
  return cudaErrorNotSupported;
}
template cudaError_t launch_fine_cg_reg<double>(cudaStream_t, const FineDev&, const double*, const double*,
                                                const double*, double, double*, double*, double*, double*, GridSync,
                                                double, int, PcgResult*);
template cudaError_t launch_fine_cg_pipe<double>(cudaStream_t, const FineDev&, const double*, const double*,
                                                 const double*, double, double*, double*, double*, double*, double*,
                                                 double*, double*, double*, double*, GridSync, double, int,
                                                 PcgResult*);
template cudaError_t launch_fine_cg<double>(cudaStream_t, const FineDev&, const double*, const double*,
                                            const double*, double, double*, double*, double*, double*, double*,
                                            double*, double*, GridSync, double, int, PcgResult*);
template cudaError_t launch_fine_cg<float>(cudaStream_t, const FineDev&, const float*, const double*, const double*,
                                           double, double*, float*, float*, float*, float*, float*, double*,
                                           GridSync, double, int, PcgResult*);


template <class T>
cudaError_t launch_coarse_step(cudaStream_t st, const LevelDev& L, const T* Hc, const T* Sinv,
                               const CoarseStepBufs<T>& B, const CoarseStepParams& P, double* partial, GridSync gs,
                               CoarseStepResult* res, bool* sell) {
  // lanes per lambda in the memory-resident loop: at least 4 (each reads a quarter of the ~14-entry rows, so the
  // group's loads of a row are coalesced and its chain of dependent loads short; measured on the 128^3 workload's
  // first coarse level, 229,538 lambdas: 164 us per iteration with 1 lane, 83 with 4, 123 with 8), and more on small
  // levels, so that they still occupy every SM
  int gsz = 4;
  while (gsz < 32 && (long)L.nlam * gsz < 65536) gsz *= 2;
  long items = (long)L.nlam * gsz;
  for (long v : {(long)L.nif, (long)L.nyl, (long)L.np, (long)L.nflux + L.np, (long)L.nc})
    if (v > items) items = v;
  const void* fn = (const void*)kp_coarse_step<T>;
  int grid = coop_grid(fn, (int)items, gs.sm_cap);
  // register-resident pipelined hybridized CG when every lambda gets its own lane group in one pass of the grid:
  // the largest power-of-two group (<= 32 lanes) that fits
  int gsz_reg = 0;
  const long lanes = (long)grid * kPThreads;
  if (L.nlam > 0 && L.nlam <= lanes) {
    gsz_reg = 1;
    while (gsz_reg < 32 && (long)L.nlam * gsz_reg * 2 <= lanes) gsz_reg *= 2;
  }
  if (sell) *sell = B.pipe.w && gsz_reg == 0 && B.hsv && L.hs_n > 0;
  void* args[] = {(void*)&L, (void*)&Hc, (void*)&Sinv, (void*)&B, (void*)&P, (void*)&partial, (void*)&gs,
                  (void*)&gsz, (void*)&gsz_reg, (void*)&res};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}
template cudaError_t launch_coarse_step<double>(cudaStream_t, const LevelDev&, const double*, const double*,
                                                const CoarseStepBufs<double>&, const CoarseStepParams&, double*,
                                                GridSync, CoarseStepResult*, bool*);

// ---- failure detection: the bounded grid barrier on its own ---------------------------------------------------
// Every block except `absent` waits at one grid barrier whose spin limit is `spin_limit` (1024-spin granularity);
// the absent block returns without arriving, so the others give up once the limit is spent, set *gs.err and leave.
// With absent < 0 every block arrives and the barrier completes. *passed counts the blocks whose wait completed.
__global__ void __launch_bounds__(kPThreads) kp_barrier_probe(GridSync gs, double* partial, int absent,
                                                              unsigned long long spin_limit, int* passed) {
  __shared__ double sm[kSmDoubles];
  Grid g{gs, partial, sm, 0u};
  if ((int)blockIdx.x == absent) return;
  const bool ok = grid_barrier(g, spin_limit);
  if (ok && threadIdx.x == 0) atomicAdd(passed, 1);
}

cudaError_t launch_barrier_probe(cudaStream_t st, GridSync gs, double* partial, int blocks, int absent,
                                 unsigned long long spin_limit, int* passed) {
  const void* fn = (const void*)kp_barrier_probe;
  const int grid = coop_grid(fn, blocks * kPThreads, gs.sm_cap);
  void* args[] = {(void*)&gs, (void*)&partial, (void*)&absent, (void*)&spin_limit, (void*)&passed};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}

}  // namespace nlmg
