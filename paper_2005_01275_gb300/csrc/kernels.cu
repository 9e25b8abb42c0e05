// Device kernels of the FAS path (sm_103a, FP64). See kernels.cuh for the data layout.
//
// All kernels are memory-bound sparse or per-cell work with little arithmetic per byte; on this part FP64 ALU
// throughput is low, so each kernel does the minimum FP64 work: kappa is evaluated once per cell (k_kappa) and read
// back by the residual, and the Picard steps freeze the face transmissibilities once (k_residual with Tval) so
// that the CG iterations only stream the frozen matrix.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "kernels.cuh"

namespace nlmg {

namespace {


template <bool MAX>
__device__ __forceinline__ double comb(double x, double y) {
  return MAX ? fmax(x, y) : x + y;
}

// Fixed-order block reduction of NV values; result in thread 0.
template <int NV, bool MAX>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] = comb<MAX>(v[k], __shfl_down_sync(0xffffffffu, v[k], off));
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[k] = comb<MAX>(v[k], __shfl_down_sync(0xffffffffu, v[k], off));
    }
  }
  __syncthreads();
}

// Grid-wide deterministic reduction; returns true in the last block (thread 0 then holds the result in v, which is
// also stored to red.out[0..NV)).
template <int NV, bool MAX>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], const Reduce& red) {
  __shared__ double sm[NV * 32];
  __shared__ int am_last;
  block_reduce<NV, MAX>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red.partial[blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(red.counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = comb<MAX>(acc[k], __ldcg(&red.partial[b * NV + k]));
  block_reduce<NV, MAX>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      red.out[k] = acc[k];
      v[k] = acc[k];
    }
    *red.counter = 0u;
  }
  return true;
}

#define GRID_STRIDE(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// ---- fine level ------------------------------------------------------------------------------------------------

__global__ void k_kappa(int n, const double* __restrict__ p, const double* __restrict__ dp, double s,
                        double* __restrict__ q, double* __restrict__ kap, double* __restrict__ dkap, int kind,
                        double a) {
  GRID_STRIDE(i, n) {
    double v = dp ? fma(s, dp[i], p[i]) : p[i];
    if (q != p) q[i] = v;
    kap[i] = kappa_of(v, kind, a);
    if (dkap) dkap[i] = dkappa_of(v, kind, a);
  }
}

__global__ void k_rhs(FineDev F, const double* __restrict__ f, const double* __restrict__ g, double* __restrict__ rhs) {
  GRID_STRIDE(K, F.N) {
    double v = F.vol[K] * f[K];
    for (int e = F.neu_off[K]; e < F.neu_off[K + 1]; ++e) v = fma(F.neu_area[e], g[F.neu_face[e]], v);
    rhs[K] = v;
  }
}

// R_K = sum_faces Ups_f (q_K - q_L) + sum_Dirichlet kappa_K Ups_K (q_K - g) - [f]_K  (eqs. TPFA_flux, FV_matrix)
// Optionally: frozen matrix entries Tval (= Ups_f), its diagonal diagT and inverse, and the exact Jacobian diagonal.
__global__ void __launch_bounds__(kThreads) k_residual(FineDev F, const double* __restrict__ q,
                                                       const double* __restrict__ kap,
                                                       const double* __restrict__ dkap,
                                                       const double* __restrict__ g,
                                                       const double* __restrict__ rhs, double* __restrict__ R,
                                                       double* __restrict__ Tval, double* __restrict__ dinv,
                                                       double* __restrict__ diagT, double* __restrict__ jdiag,
                                                       double* __restrict__ Joff, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(K, F.N) {
    const double qK = q[K], kK = kap[K];
    const double dkK = jdiag ? dkap[K] : 0.0;
    double flux = 0.0, dsum = 0.0, jd = 0.0;
    const int w = F.sell_w[K >> 5];
    int e = F.sell_off[K >> 5] + (K & 31);
    for (int j = 0; j < w; ++j, e += 32) {
      const int L = F.nbr[e];
      const double us = F.ups_s[e];
      const double ha = kK * us, hb = kap[L] * F.ups_n[e];
      const double t = hb / (ha + hb);           // Ups / ha
      const double T = ha * t;                   // harmonic mean of the two kappa-scaled halves
      const double diff = qK - q[L];
      flux = fma(T, diff, flux);
      dsum += T;
      if (Tval) Tval[e] = T;
      if (jdiag) jd += T + t * t * dkK * us * diff;
      // dR_K/dp_L = -Ups + (Ups/hb)^2 kappa'(p_L) Ups_bar_L (p_K - p_L), Ups/hb = ha / (ha + hb)
      if (Joff) {
        const double tb = ha / (ha + hb);
        Joff[e] = -T + tb * tb * dkap[L] * F.ups_n[e] * diff;
      }
    }
    for (int e = F.dir_off[K]; e < F.dir_off[K + 1]; ++e) {
      const double h = kK * F.dir_ups[e];
      const double diff = qK - g[F.dir_face[e]];
      flux = fma(h, diff, flux);
      dsum += h;
      if (jdiag) jd += dkK * F.dir_ups[e] * diff + h;
    }
    const double r = flux - rhs[K];
    R[K] = r;
    acc[0] = fma(r, r, acc[0]);
    if (diagT) diagT[K] = dsum;
    if (dinv) dinv[K] = 1.0 / dsum;
    if (jdiag) jdiag[K] = jd;
  }
  grid_reduce<1, false>(acc, red);
}

// S = diag(A)^-1/2 of the frozen matrix, then the scaled off-diagonal entries Ts = S_K T S_L (SELL layout)
__global__ void k_sdiag(int n, const double* __restrict__ diagT, double* __restrict__ sdiag) {
  GRID_STRIDE(i, n) sdiag[i] = 1.0 / sqrt(diagT[i]);
}

template <class T>
__global__ void k_scale_sell(FineDev F, const double* __restrict__ Tval, const double* __restrict__ sdiag,
                             T* __restrict__ Ts) {
  GRID_STRIDE(K, F.N) {
    const int w = F.sell_w[K >> 5];
    const double sK = sdiag[K];
    int e = F.sell_off[K >> 5] + (K & 31);
    for (int j = 0; j < w; ++j, e += 32) Ts[e] = (T)(Tval[e] * sK * sdiag[F.nbr[e]]);
  }
}

__global__ void k_jacobi_update(int n, const double* __restrict__ q, const double* __restrict__ R,
                                const double* __restrict__ jdiag, const double* __restrict__ diagT, double omega,
                                double* __restrict__ qnew) {
  GRID_STRIDE(i, n) {
    double d = fmax(jdiag[i], 0.5 * diagT[i]);
    qnew[i] = q[i] - omega * R[i] / d;
  }
}

__global__ void k_max_abs(int n, const double* __restrict__ x, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(i, n) acc[0] = fmax(acc[0], fabs(x[i]));
  grid_reduce<1, true>(acc, red);
}

__global__ void k_axpy(int n, const double* __restrict__ x, double s, const double* __restrict__ dx,
                       double* __restrict__ out) {
  GRID_STRIDE(i, n) out[i] = fma(s, dx[i], x[i]);
}

__global__ void k_sub(int n, const double* __restrict__ y, const double* __restrict__ x, double* __restrict__ out) {
  GRID_STRIDE(i, n) out[i] = y[i] - x[i];
}

// TPFA flux on each level-0 flux unknown, oriented out of K (eq. TPFA_flux).
__global__ void k_fine_flux(FineDev F, const double* __restrict__ p, const double* __restrict__ kap,
                            const double* __restrict__ g, double* __restrict__ sigma) {
  GRID_STRIDE(j, F.nflux) {
    const int K = F.fl_k[j], L = F.fl_l[j];
    const double ha = kap[K] * F.fl_u0[j];
    double s;
    if (L >= 0) {
      const double hb = kap[L] * F.fl_u1[j];
      const double T = ha * (hb / (ha + hb));
      s = T * (p[K] - p[L]);
    } else {
      s = ha * (p[K] - g[F.fl_face[j]]);
    }
    sigma[j] = s;
  }
}

// ---- GMRES helpers (single-level Newton baseline) ---------------------------------------------------------------

// w = J (dinv .* v) with J = jdiag on the diagonal and Joff off it (SELL layout): the right-preconditioned operator
__global__ void k_jac_apply(FineDev F, const double* __restrict__ jdiag, const double* __restrict__ Joff,
                            const double* __restrict__ dinv, const double* __restrict__ v, double* __restrict__ w) {
  GRID_STRIDE(K, F.N) {
    double y = jdiag[K] * dinv[K] * v[K];
    const int wdt = F.sell_w[K >> 5];
    int e = F.sell_off[K >> 5] + (K & 31);
    for (int j = 0; j < wdt; ++j, e += 32) {
      const int L = F.nbr[e];
      y = fma(Joff[e], dinv[L] * v[L], y);
    }
    w[K] = y;
  }
}

// h[k] = V_k . w for k < nk (V stored as nk consecutive vectors of length n); fixed-order grid reduction per k
__global__ void k_mdot(int n, int nk, const double* __restrict__ V, const double* __restrict__ w, double* partial,
                       unsigned* counter, double* h) {
  __shared__ double sm[32];
  __shared__ int am_last;
  for (int k = 0; k < nk; ++k) {
    double acc[1] = {0.0};
    const double* Vk = V + (size_t)k * n;
    GRID_STRIDE(i, n) acc[0] = fma(Vk[i], w[i], acc[0]);
    block_reduce<1, false>(acc, sm);
    if (threadIdx.x == 0) partial[(size_t)k * gridDim.x + blockIdx.x] = acc[0];
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  for (int k = 0; k < nk; ++k) {
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc[0] += __ldcg(&partial[(size_t)k * gridDim.x + b]);
    block_reduce<1, false>(acc, sm);
    if (threadIdx.x == 0) h[k] = acc[0];
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// w -= sum_k h[k] V_k ; then the norm of the result (grid reduction into red.out)
__global__ void k_orth_update(int n, int nk, const double* __restrict__ V, const double* __restrict__ h,
                              double* __restrict__ w, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(i, n) {
    double v = w[i];
    for (int k = 0; k < nk; ++k) v = fma(-h[k], V[(size_t)k * n + i], v);
    w[i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  grid_reduce<1, false>(acc, red);
}

__global__ void k_scale_vec(int n, const double* __restrict__ x, double s, double* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = s * x[i];
}

// x = dinv .* (sum_k y[k] V_k)   (dinv may be null: no scaling)
__global__ void k_gmres_combine(int n, int nk, const double* __restrict__ V, const double* __restrict__ y,
                                const double* __restrict__ dinv, double* __restrict__ x) {
  GRID_STRIDE(i, n) {
    double v = 0.0;
    for (int k = 0; k < nk; ++k) v = fma(y[k], V[(size_t)k * n + i], v);
    x[i] = dinv ? dinv[i] * v : v;
  }
}

// Jacobi scaling of the Newton system, with the same safeguard as the Jacobi smoother: 1 / max(J_KK, d_K / 2)
__global__ void k_jacobi_dinv(int n, const double* __restrict__ jdiag, const double* __restrict__ diagT,
                              double* __restrict__ out) {
  GRID_STRIDE(i, n) out[i] = 1.0 / fmax(jdiag[i], 0.5 * diagT[i]);
}

// Scaled Newton system of the level-0 BiCGStab: with D = jdinv = 1 / max(J_KK, d_K / 2) and S = D^1/2,
// sS = S, jd = J_KK D_K on the diagonal and Js = S_K J_KL S_L off it (SELL layout; padding entries stay 0).
__global__ void k_scale_jac(FineDev F, const double* __restrict__ jdiag, const double* __restrict__ Joff,
                            const double* __restrict__ jdinv, double* __restrict__ Js, double* __restrict__ jd,
                            double* __restrict__ sS) {
  GRID_STRIDE(K, F.N) {
    const double sK = sqrt(jdinv[K]);
    sS[K] = sK;
    jd[K] = jdiag[K] * jdinv[K];
    const int w = F.sell_w[K >> 5];
    int e = F.sell_off[K >> 5] + (K & 31);
    for (int j = 0; j < w; ++j, e += 32) Js[e] = Joff[e] * sK * sqrt(jdinv[F.nbr[e]]);
  }
}

// ---- measurement: FP64 FMA throughput (8 independent dependency chains per thread) ----------------------------
__global__ void k_fp64_peak(int iters, double* out) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-7 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 0.9999999, 1e-9);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---- transfers -------------------------------------------------------------------------------------------------

// out1 = scale1 * P_A^T in1 (and out2 = P_A^T in2) per aggregate: one warp per aggregate, fixed-order warp sums.
__global__ void k_restrict_p(TransferDev T, const double* __restrict__ in1, double* __restrict__ out1,
                             double scale1, const double* __restrict__ in2, double* __restrict__ out2) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int a = warp; a < T.na; a += nwarps) {
    const int ma = T.mc[a], r0 = T.rows_off[a], r1 = T.rows_off[a + 1];
    const double* P = T.Pblk + T.pblk_off[a];
    double s1[kMaxM], s2[kMaxM];
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) s1[j] = s2[j] = 0.0;
    for (int t = r0 + lane; t < r1; t += 32) {
      const int idx = T.rows[t];
      const double v1 = in1[idx];
      const double v2 = in2 ? in2[idx] : 0.0;
      const double* Pr = P + (size_t)(t - r0) * ma;
#pragma unroll
      for (int j = 0; j < kMaxM; ++j)
        if (j < ma) {
          s1[j] = fma(Pr[j], v1, s1[j]);
          s2[j] = fma(Pr[j], v2, s2[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxM; ++j)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1[j] += __shfl_xor_sync(0xffffffffu, s1[j], off);
        s2[j] += __shfl_xor_sync(0xffffffffu, s2[j], off);
      }
    if (lane == 0)
      for (int j = 0; j < ma; ++j) {
        out1[T.pc_off[a] + j] = scale1 * s1[j];
        if (out2) out2[T.pc_off[a] + j] = s2[j];
      }
  }
}

__global__ void k_prolong_p(TransferDev T, const double* __restrict__ e, double* __restrict__ out) {
  GRID_STRIDE(i, T.nrows) {
    const int a = T.pd_agg[i], t = T.pd_row[i], ma = T.mc[a];
    const double* Pr = T.Pblk + T.pblk_off[a] + (size_t)t * ma;
    const double* ea = e + T.pc_off[a];
    double v = 0.0;
    for (int j = 0; j < ma; ++j) v = fma(Pr[j], ea[j], v);
    out[i] = v;
  }
}

// y = alpha A x + beta y for a CSR matrix (the sparse transfers): kCsrLanes adjacent lanes per row, each taking every
// kCsrLanes-th entry, then a fixed shuffle tree (the rows are short and the level is small, so spreading a row
// over lanes hides the gather latency that a thread per row would serialise). Warp-uniform loop: every lane takes
// part in the shuffles.
constexpr int kCsrLanes = 4;
__global__ void k_csr(int nrows, const int* __restrict__ off, const int* __restrict__ col,
                      const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                      double alpha, double beta) {
  const long total = (long)nrows * kCsrLanes;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long tb = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); tb < total; tb += stride) {
    const long t = tb + lane;
    const bool act = t < total;
    const int r = act ? (int)(t / kCsrLanes) : 0;
    const int g = (int)(t & (kCsrLanes - 1));
    double v = 0.0;
    if (act)
      for (int k = off[r] + g; k < off[r + 1]; k += kCsrLanes) v = fma(val[k], x[col[k]], v);
#pragma unroll
    for (int o = kCsrLanes >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (act && g == 0) y[r] = beta == 0.0 ? alpha * v : fma(beta, y[r], alpha * v);
  }
}

// ---- coarse levels ---------------------------------------------------------------------------------------------

// Coarse operator (Prop. 1, eq. structure) on cell c: pbar = w_c . p_c, s = 1 / kappa(pbar);
// yl[slots of c] = s Mloc_c sigma_c + Dloc_c^T p_c (one thread per local flux slot) and
// r_p,c = Dloc_c sigma_c - b_p,c (one thread per pressure unknown).
__global__ void k_coarse_kappa(LevelDev L, const double* __restrict__ p, double* __restrict__ kapc, int kind,
                               double a) {
  GRID_STRIDE(c, L.nc) {
    const int po = L.p_off[c];
    double pb = 0.0;
    for (int r = 0; r < L.m[c]; ++r) pb = fma(L.w[po + r], p[po + r], pb);
    kapc[c] = kappa_of(pb, kind, a);
  }
}

__global__ void k_coarse_slots(LevelDev L, const double* __restrict__ sig, const double* __restrict__ p,
                               const double* __restrict__ kapc, double* __restrict__ yl) {
  GRID_STRIDE(y, L.nyl) {
    const int c = L.slot_cell[y];
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c];
    const int u = y - lo;
    const double* Mu = L.Mloc + L.mat_off[c] + (size_t)u * nl;
    const double* D = L.Dloc + L.dmat_off[c];
    double acc = 0.0;
    for (int t = 0; t < nl; ++t) acc = fma(Mu[t], sig[L.loc[lo + t]], acc);
    acc /= kapc[c];
    for (int r = 0; r < mc; ++r) acc = fma(D[r * nl + u], p[po + r], acc);
    yl[y] = acc;
  }
}

__global__ void k_coarse_prows(LevelDev L, const double* __restrict__ sig, const double* __restrict__ bp,
                               double* __restrict__ rp, Reduce red) {
  double acc2[1] = {0.0};
  GRID_STRIDE(i, L.np) {
    const int c = L.p_cell[i];
    const int lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c];
    const double* Dr = L.Dloc + L.dmat_off[c] + (size_t)(i - po) * nl;
    double v = 0.0;
    for (int t = 0; t < nl; ++t) v = fma(Dr[t], sig[L.loc[lo + t]], v);
    if (bp) v -= bp[i];
    rp[i] = v;
    acc2[0] = fma(v, v, acc2[0]);
  }
  grid_reduce<1, false>(acc2, red);
}

// r_sigma,i = (sum over the <= 2 owners of yl) - b_sigma,i
__global__ void k_coarse_flux(LevelDev L, const double* __restrict__ yl, const double* __restrict__ bs,
                              double* __restrict__ rs, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(i, L.nflux) {
    double v = yl[L.f_y0[i]];
    if (L.f_y1[i] >= 0) v += yl[L.f_y1[i]];
    if (bs) v -= bs[i];
    rs[i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  grid_reduce<1, false>(acc, red);
}

__global__ void k_coarse_pbar_max(LevelDev L, const double* __restrict__ dp, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(c, L.nc) {
    const int po = L.p_off[c];
    double v = 0.0;
    for (int r = 0; r < L.m[c]; ++r) v = fma(L.w[po + r], dp[po + r], v);
    acc[0] = fmax(acc[0], fabs(v));
  }
  grid_reduce<1, true>(acc, red);
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------------------------------------

static std::atomic<long long> g_launches(0);
static thread_local long long t_launches = 0;   // launches issued by the calling host thread
long long launch_count() { return g_launches.load(); }
long long launch_count_thread() { return t_launches; }
void count_launch(int n) {
  g_launches.fetch_add(n);
  t_launches += n;
}
#define COUNT(n) count_launch(n)

void launch_kappa(cudaStream_t st, int n, const double* p, const double* dp, double s, double* q, double* kap,
                  double* dkap, int kind, double a) {
  COUNT(1);
  k_kappa<<<grid_for(n), kThreads, 0, st>>>(n, p, dp, s, q, kap, dkap, kind, a);
}
void launch_rhs(cudaStream_t st, const FineDev& F, const double* f, const double* g, double* rhs) {
  COUNT(1);
  k_rhs<<<grid_for(F.N), kThreads, 0, st>>>(F, f, g, rhs);
}
void launch_residual(cudaStream_t st, const FineDev& F, const double* q, const double* kap, const double* dkap,
                     const double* g, const double* rhs, double* R, double* Tval, double* dinv, double* diagT,
                     double* jdiag, Reduce red, double* Joff) {
  COUNT(1);
  k_residual<<<grid_for(F.N), kThreads, 0, st>>>(F, q, kap, dkap, g, rhs, R, Tval, dinv, diagT, jdiag, Joff, red);
}
void launch_jacobi_update(cudaStream_t st, int n, const double* q, const double* R, const double* jdiag,
                          const double* diagT, double omega, double* qnew) {
  COUNT(1);
  k_jacobi_update<<<grid_for(n), kThreads, 0, st>>>(n, q, R, jdiag, diagT, omega, qnew);
}
void launch_max_abs(cudaStream_t st, int n, const double* x, Reduce red) {
  COUNT(1);
  k_max_abs<<<grid_for(n), kThreads, 0, st>>>(n, x, red);
}
void launch_axpy(cudaStream_t st, int n, const double* x, double s, const double* dx, double* out) {
  COUNT(1);
  k_axpy<<<grid_for(n), kThreads, 0, st>>>(n, x, s, dx, out);
}
void launch_sub(cudaStream_t st, int n, const double* y, const double* x, double* out) {
  COUNT(1);
  k_sub<<<grid_for(n), kThreads, 0, st>>>(n, y, x, out);
}
void launch_fine_flux(cudaStream_t st, const FineDev& F, const double* p, const double* kap, const double* g,
                      double* sigma) {
  COUNT(1);
  k_fine_flux<<<grid_for(F.nflux), kThreads, 0, st>>>(F, p, kap, g, sigma);
}
void launch_restrict_p(cudaStream_t st, const TransferDev& T, const double* in1, double* out1, double scale1,
                       const double* in2, double* out2) {
  COUNT(1);
  long threads = (long)T.na * 32;
  k_restrict_p<<<grid_for(threads), kThreads, 0, st>>>(T, in1, out1, scale1, in2, out2);
}
void launch_prolong_p(cudaStream_t st, const TransferDev& T, const double* e, double* out) {
  COUNT(1);
  k_prolong_p<<<grid_for(T.nrows), kThreads, 0, st>>>(T, e, out);
}
void launch_csr(cudaStream_t st, int nrows, const int* off, const int* col, const double* val, const double* x,
                double* y, double alpha, double beta) {
  COUNT(1);
  k_csr<<<grid_for((long)nrows * kCsrLanes), kThreads, 0, st>>>(nrows, off, col, val, x, y, alpha, beta);
}
void launch_coarse_cell(cudaStream_t st, const LevelDev& L, const double* sig, const double* p, const double* bp,
                        double* yl, double* rp, double* kapc, int kind, double a, Reduce red) {
  COUNT(3);
  k_coarse_kappa<<<grid_for(L.nc), kThreads, 0, st>>>(L, p, kapc, kind, a);
  k_coarse_slots<<<grid_for(L.nyl), kThreads, 0, st>>>(L, sig, p, kapc, yl);
  k_coarse_prows<<<grid_for(L.np), kThreads, 0, st>>>(L, sig, bp, rp, red);
}
void launch_jac_apply(cudaStream_t st, const FineDev& F, const double* jdiag, const double* Joff,
                      const double* dinv, const double* v, double* w) {
  COUNT(1);
  k_jac_apply<<<grid_for(F.N), kThreads, 0, st>>>(F, jdiag, Joff, dinv, v, w);
}
void launch_mdot(cudaStream_t st, int n, int nk, const double* V, const double* w, double* partial,
                 unsigned* counter, double* h) {
  COUNT(1);
  k_mdot<<<std::min(grid_for(n), 256), kThreads, 0, st>>>(n, nk, V, w, partial, counter, h);
}
void launch_orth_update(cudaStream_t st, int n, int nk, const double* V, const double* h, double* w, Reduce red) {
  COUNT(1);
  k_orth_update<<<grid_for(n), kThreads, 0, st>>>(n, nk, V, h, w, red);
}
void launch_scale_vec(cudaStream_t st, int n, const double* x, double s, double* y) {
  COUNT(1);
  k_scale_vec<<<grid_for(n), kThreads, 0, st>>>(n, x, s, y);
}
void launch_gmres_combine(cudaStream_t st, int n, int nk, const double* V, const double* y, const double* dinv,
                          double* x) {
  COUNT(1);
  k_gmres_combine<<<grid_for(n), kThreads, 0, st>>>(n, nk, V, y, dinv, x);
}
void launch_jacobi_dinv(cudaStream_t st, int n, const double* jdiag, const double* diagT, double* out) {
  COUNT(1);
  k_jacobi_dinv<<<grid_for(n), kThreads, 0, st>>>(n, jdiag, diagT, out);
}
void launch_scale_jac(cudaStream_t st, const FineDev& F, const double* jdiag, const double* Joff,
                      const double* jdinv, double* Js, double* jd, double* sS) {
  COUNT(1);
  k_scale_jac<<<grid_for(F.N), kThreads, 0, st>>>(F, jdiag, Joff, jdinv, Js, jd, sS);
}
bool measure_fp64_peak(double* gflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 8192;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_peak<<<blocks, threads>>>(iters / 8, out);   // warm-up
  cudaEventRecord(e0);
  k_fp64_peak<<<blocks, threads>>>(iters, out);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  COUNT(2);
  *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e9;
  return cudaGetLastError() == cudaSuccess;
}
void launch_sdiag(cudaStream_t st, int n, const double* diagT, double* sdiag) {
  COUNT(1);
  k_sdiag<<<grid_for(n), kThreads, 0, st>>>(n, diagT, sdiag);
}
template <class T>
void launch_scale_sell(cudaStream_t st, const FineDev& F, const double* Tval, const double* sdiag, T* Ts) {
  COUNT(1);
  k_scale_sell<T><<<grid_for(F.N), kThreads, 0, st>>>(F, Tval, sdiag, Ts);
}
template void launch_scale_sell<double>(cudaStream_t, const FineDev&, const double*, const double*, double*);
template void launch_scale_sell<float>(cudaStream_t, const FineDev&, const double*, const double*, float*);
void launch_coarse_flux(cudaStream_t st, const LevelDev& L, const double* yl, const double* bs, double* rs,
                        Reduce red) {
  COUNT(1);
  k_coarse_flux<<<grid_for(L.nflux), kThreads, 0, st>>>(L, yl, bs, rs, red);
}
void launch_coarse_pbar_max(cudaStream_t st, const LevelDev& L, const double* dp, Reduce red) {
  COUNT(1);
  k_coarse_pbar_max<<<grid_for(L.nc), kThreads, 0, st>>>(L, dp, red);
}

}  // namespace nlmg
