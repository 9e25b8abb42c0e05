// Persistent (cooperative) conjugate-gradient kernels: one launch runs a whole Picard linear solve, with
// device-side scalars and convergence test, so the CG iterations pay neither launch gaps nor host round trips.
//
// Grid-wide synchronisation uses a counter/generation barrier whose wait is bounded: after ~2 s of spinning the
// kernel records an error flag and every block leaves. The launch goes through cudaLaunchCooperativeKernel with at
// most the co-resident number of blocks, so in a correct run every wait ends.
//
// Data written by one block and read by another inside the same launch (CG vectors, per-interface buffers) is read
// with ld.global.cg (L2, bypassing the non-coherent L1), after the barrier that orders the write.
//
// Reductions stay deterministic: each block writes one partial; the last block to reach the barrier sums them in
// block order with a fixed tree and derives the step lengths once, and every block reads the same scalars, so all
// blocks take the same decisions and a run is bitwise reproducible.
#include <cmath>

#include "kernels.cuh"
#include "persist.cuh"

namespace nlmg {

namespace {

constexpr unsigned long long kSpinLimit = 1ull << 26;   // x ~32 ns sleeps ~ 2 s
constexpr int kPThreads = 512;                           // threads per block of the persistent kernels

// Bounded grid barrier: blocks arrive on gs.count; the last one to arrive runs `last` (a block-wide callback),
// then bumps the generation that the others poll. Returns false (and sets *err) if a wait gave up.
template <class LastFn>
__device__ __forceinline__ bool grid_barrier_ex(const GridSync& gs, LastFn&& last) {
  __shared__ int ok, is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = gs.gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(gs.count, 1u);
    is_last = arrived == gridDim.x - 1;
    if (!is_last) {
      unsigned long long spins = 0;
      while (*gen == g) {
        __nanosleep(32);
        if ((++spins & 1023u) == 0 && (spins > kSpinLimit || *((volatile int*)gs.err) != 0)) {
          atomicExch(gs.err, 1);
          ok = 0;
          break;
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    last();
    __syncthreads();
    if (threadIdx.x == 0) {
      *gs.count = 0u;
      __threadfence();
      atomicAdd(gs.gen, 1u);
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ bool grid_barrier(const GridSync& gs) {
  return grid_barrier_ex(gs, []() {});
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) sm[k * 32] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sm[k * 32];
  __syncthreads();
}

// Grid sums of NV values: every block publishes its block sum; the last block to arrive adds the partials in block
// order (fixed tree) and stores the result to out[0..NV-1]; its thread 0 then runs `post(out)`, which derives NX
// scalars from the sums (the CG step lengths) into out[NV..NV+NX-1], so that each division is done once per grid
// instead of once per thread. After the barrier every thread reads all NV + NX values.
template <int NV, int NX = 0, class PostFn>
__device__ __forceinline__ bool grid_sum_x(double (&v)[NV + NX], double* partial, double* out, const GridSync& gs,
                                           double* sm, PostFn&& post) {
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) w[k] = v[k];
  block_sum<NV>(w, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) partial[blockIdx.x * NV + k] = w[k];
  const bool ok = grid_barrier_ex(gs, [&]() {
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partial[b * NV + k]);
    block_sum<NV>(acc, sm);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) out[k] = acc[k];
      post(out);
    }
    __threadfence();
  });
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k < NV + NX; ++k) v[k] = __ldcg(&out[k]);
  return true;
}

template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partial, double* out, const GridSync& gs,
                                         double* sm) {
  return grid_sum_x<NV, 0>(v, partial, out, gs, sm, [](double*) {});
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
  __shared__ double sm[2 * 32];
  double* part0 = partial;
  double* part1 = partial + 2 * gridDim.x;
  T t1 = (T)0;   // per-thread partial sums in T (a thread holds one or two cells), block and grid sums in FP64
  GSTRIDE(i, F.N) {
    const T ri = (T)(sdiag[i] * bscale * b[i]);
    y[i] = (T)0;
    r[i] = ri;
    t1 = fma(ri, ri, t1);
  }
  double a1[1] = {(double)t1};
  if (!grid_sum<1>(a1, part1, gs.out + 0, gs, sm)) return;
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
    if (!grid_sum_x<1, 1>(pq, part0, gs.out + 8, gs, sm, [&](double* o) { o[1] = o[0] != 0.0 ? rr / o[0] : 0.0; }))
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
    if (!grid_sum_x<1, 1>(rn, part1, gs.out + 16, gs, sm, [&](double* o) { o[1] = rr != 0.0 ? o[0] / rr : 0.0; }))
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
  __shared__ double sm[2 * 32];
  double* part0 = partial;
  double* part1 = partial + 2 * gridDim.x;
  GSTRIDE(i, F.N) {
    r[i] = (T)(sdiag[i] * bscale * b[i]);
    y[i] = z[i] = sv[i] = p[i] = (T)0;
  }
  if (!grid_barrier(gs)) return;
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
  if (!grid_sum_x<2, 2>(a4, part1, gs.out + 0, gs, sm, [&](double* o) {
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
    if (!grid_sum_x<2, 2>(n4, (it & 1) ? part1 : part0, gs.out + ((it & 1) ? 16 : 8), gs, sm, [&](double* o) {
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

// ---- coarse level: hybridized saddle solve (rhs, Jacobi diagonal, CG on H lambda = xi, local recovery) ------
template <class T>
__global__ void __launch_bounds__(kPThreads) kp_hyb_solve(LevelDev L, const T* __restrict__ Hc,
                                                         const T* __restrict__ Sinv,
                                                         const double* __restrict__ kapc,
                                                         const double* __restrict__ bs,
                                                         const double* __restrict__ bp, T* ylam,
                                                         T* ydiag, T* lam, T* lr, T* lz,
                                                         T* pa, T* pb, T* lq, T* ldinv,
                                                         double* __restrict__ dsig, double* __restrict__ dp,
                                                         double* partial, GridSync gs, double tol, int maxit,
                                                         int gsz, PcgResult* res) {
  __shared__ double sm[2 * 32];
  double* part0 = partial;
  double* part1 = partial + 2 * gridDim.x;
  // phase 0: per interface slot k of cell c, u_k = kappa A[k,:] bhat + B[k,:] b_p (signed) and kappa Hc[k,k]
  GSTRIDE(k, L.nif) {
    const int c = L.if_cell[k];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const double kp = kapc[c];
    const int u = L.if_slot[k];
    const T* Su = Sinv + L.sad_off[c] + (size_t)u * n;
    T a1 = 0, a2_ = 0;
    for (int t = 0; t < nl; ++t)
      if (L.own0[lo + t]) a1 += Su[t] * (T)bs[L.loc[lo + t]];
    for (int q = 0; q < mc; ++q) a2_ += Su[nl + q] * (T)bp[po + q];
    ylam[k] = (T)L.if_sign[k] * ((T)kp * a1 + a2_);
    const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
    ydiag[k] = (T)kp * Hc[L.hc_off[c] + (k - k0) * ni + (k - k0)];
  }
  if (!grid_barrier(gs)) return;
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
  if (!grid_sum<2>(a2, part1, gs.out + 0, gs, sm)) return;
  double rz = a2[0];
  const double rr0 = a2[1];
  double rr = rr0;
  const double tol2 = tol * tol * rr0;
  T beta = (T)0;
  T* pp = pa;       // search direction p
  int it = 0;
  while (rr0 > 0.0 && rr > tol2 && it < maxit) {
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
            hz += (T)kapc[c] * y;
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
    if (!grid_sum_x<1, 1>(a1, part0, gs.out + 8, gs, sm, [&](double* o) { o[1] = o[0] != 0.0 ? rz / o[0] : 0.0; }))
      return;
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
    if (!grid_sum_x<2, 1>(a3, part1, gs.out + 16, gs, sm,
                          [&](double* o) { o[2] = rz != 0.0 ? o[0] / rz : 0.0; }))
      return;
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
      if (L.own0[lo + t]) a1 += Su[t] * (T)bs[L.loc[lo + t]];
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k)
      a1 -= Su[L.if_slot[k]] * (T)L.if_sign[k] * __ldcg(&lam[L.if_lam[k]]);
    for (int q = 0; q < mc; ++q) a2_ += Su[nl + q] * (T)bp[po + q];
    dsig[L.loc[y]] = (double)((T)kapc[c] * a1 + a2_);
  }
  GSTRIDE(i, L.np) {
    const int c = L.p_cell[i];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const T* Sr = Sinv + L.sad_off[c] + (size_t)(nl + i - po) * n;
    T a1 = 0, a2_ = 0;
    for (int t = 0; t < nl; ++t)
      if (L.own0[lo + t]) a1 += Sr[t] * (T)bs[L.loc[lo + t]];
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k)
      a1 -= Sr[L.if_slot[k]] * (T)L.if_sign[k] * __ldcg(&lam[L.if_lam[k]]);
    for (int q = 0; q < mc; ++q) a2_ += Sr[nl + q] * (T)bp[po + q];
    dp[i] = (double)a1 + (double)a2_ / kapc[c];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res->iters = it;
    res->rr0 = rr0;
    res->rr = rr;
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
cudaError_t launch_hyb_solve(cudaStream_t st, const LevelDev& L, const T* Hc, const T* Sinv, const double* kapc,
                             const double* bs, const double* bp, T* ylam, T* ydiag, T* lam, T* lr, T* lz, T* pa,
                             T* pb, T* lq, T* ldinv, double* dsig, double* dp, double* partial, GridSync gs,
                             double tol, int maxit, PcgResult* res) {
  // lanes per lambda in the H product: enough that the level spreads over ~64k threads
  int gsz = 1;
  while (gsz < 32 && (long)L.nlam * gsz < 65536) gsz *= 2;
  long items = (long)L.nlam * gsz;
  if (L.nif > items) items = L.nif;
  if (L.nyl > items) items = L.nyl;
  const void* fn = (const void*)kp_hyb_solve<T>;
  int grid = coop_grid(fn, (int)items, gs.sm_cap);
  void* args[] = {(void*)&L, (void*)&Hc, (void*)&Sinv, (void*)&kapc, (void*)&bs, (void*)&bp, (void*)&ylam,
                  (void*)&ydiag, (void*)&lam, (void*)&lr, (void*)&lz, (void*)&pa, (void*)&pb, (void*)&lq,
                  (void*)&ldinv, (void*)&dsig, (void*)&dp, (void*)&partial, (void*)&gs, (void*)&tol, (void*)&maxit,
                  (void*)&gsz, (void*)&res};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}
template cudaError_t launch_hyb_solve<double>(cudaStream_t, const LevelDev&, const double*, const double*,
                                              const double*, const double*, const double*, double*, double*,
                                              double*, double*, double*, double*, double*, double*, double*,
                                              double*, double*, double*, GridSync, double, int, PcgResult*);
template cudaError_t launch_hyb_solve<float>(cudaStream_t, const LevelDev&, const float*, const float*,
                                             const double*, const double*, const double*, float*, float*, float*,
                                             float*, float*, float*, float*, float*, float*, double*, double*,
                                             double*, GridSync, double, int, PcgResult*);

}  // namespace nlmg
