// Device kernels of the FAS path (sm_103a, FP64). See kernels.cuh for the data layout.
//
// All kernels are memory-bound sparse or per-cell work with little arithmetic per byte; on this part FP64 ALU
// throughput is low, so each kernel does the minimum FP64 work: kappa is evaluated once per cell (k_kappa) and read
// back by the residual, and the Picard steps freeze the face transmissibilities once (k_residual with Tval) so
// that the CG iterations only stream the frozen matrix.
#include <atomic>
#include <cmath>

#include "kernels.cuh"

namespace nlmg {

namespace {

__device__ __forceinline__ double kappa_of(double p, int kind, double a) {
  return kind == 0 ? exp(a * p) : 1.0 / (1.0 + p * p);
}
__device__ __forceinline__ double dkappa_of(double p, int kind, double a) {
  if (kind == 0) return a * exp(a * p);
  double t = 1.0 + p * p;
  return -2.0 * p / (t * t);
}

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
                                                       Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(K, F.N) {
    const double qK = q[K], kK = kap[K];
    const double dkK = jdiag ? dkap[K] : 0.0;
    double flux = 0.0, dsum = 0.0, jd = 0.0;
    const int e1 = F.row_off[K + 1];
    for (int e = F.row_off[K]; e < e1; ++e) {
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

__global__ void k_jacobi_update(int n, const double* __restrict__ q, const double* __restrict__ R,
                                const double* __restrict__ jdiag, const double* __restrict__ diagT, double omega,
                                double* __restrict__ qnew) {
  GRID_STRIDE(i, n) {
    double d = fmax(jdiag[i], 0.5 * diagT[i]);
    qnew[i] = q[i] - omega * R[i] / d;
  }
}

// CG direction update fused into the matrix product: p_new = z + beta p_old (computed for the row and its
// neighbours alike), q = A p_new, and the reduction p_new . q; the last block sets alpha = (r.z) / (p.q).
__global__ void __launch_bounds__(kThreads) k_fine_spmv(FineDev F, const double* __restrict__ Tval,
                                                        const double* __restrict__ diagT,
                                                        const double* __restrict__ z,
                                                        const double* __restrict__ pold, double* __restrict__ pnew,
                                                        double* __restrict__ q, double* sc, int first, Reduce red) {
  const double beta = first ? 0.0 : sc[S_BETA];
  double acc[1] = {0.0};
  GRID_STRIDE(K, F.N) {
    const double pK = first ? z[K] : fma(beta, pold[K], z[K]);
    double y = diagT[K] * pK;
    const int e1 = F.row_off[K + 1];
    for (int e = F.row_off[K]; e < e1; ++e) {
      const int L = F.nbr[e];
      const double pL = first ? z[L] : fma(beta, pold[L], z[L]);
      y = fma(-Tval[e], pL, y);
    }
    pnew[K] = pK;
    q[K] = y;
    acc[0] = fma(pK, y, acc[0]);
  }
  if (grid_reduce<1, false>(acc, red) && threadIdx.x == 0) {
    sc[S_PQ] = acc[0];
    sc[S_ALPHA] = acc[0] != 0.0 ? sc[S_RZ] / acc[0] : 0.0;
  }
}

__global__ void k_pcg_init(int n, const double* __restrict__ b, double bscale, const double* __restrict__ dinv,
                           double* __restrict__ x, double* __restrict__ r, double* __restrict__ z, double* sc,
                           Reduce red) {
  double acc[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    double ri = bscale * b[i];
    double zi = ri * dinv[i];
    x[i] = 0.0;
    r[i] = ri;
    z[i] = zi;
    acc[0] = fma(ri, zi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
  }
  if (grid_reduce<2, false>(acc, red) && threadIdx.x == 0) {
    sc[S_RZ] = acc[0];
    sc[S_RR0] = acc[1];
    sc[S_RR] = acc[1];
    sc[S_BETA] = 0.0;
  }
}

__global__ void k_pcg_update(int n, double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                             const double* __restrict__ p, const double* __restrict__ q,
                             const double* __restrict__ dinv, double* sc, Reduce red) {
  const double alpha = sc[S_ALPHA];
  double acc[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    acc[0] = fma(ri, zi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
  }
  if (grid_reduce<2, false>(acc, red) && threadIdx.x == 0) {
    double rz_old = sc[S_RZ];
    sc[S_BETA] = rz_old != 0.0 ? acc[0] / rz_old : 0.0;
    sc[S_RZ] = acc[0];
    sc[S_RR] = acc[1];
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

__global__ void k_csr(int nrows, const int* __restrict__ off, const int* __restrict__ col,
                      const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                      double alpha, double beta) {
  GRID_STRIDE(r, nrows) {
    double v = 0.0;
    for (int k = off[r]; k < off[r + 1]; ++k) v = fma(val[k], x[col[k]], v);
    y[r] = beta == 0.0 ? alpha * v : fma(beta, y[r], alpha * v);
  }
}

// ---- coarse levels ---------------------------------------------------------------------------------------------

// Per coarse cell c (Prop. 1, eq. structure): pbar = w_c . p_c, s = 1 / kappa(pbar);
// yl[slots of c] = s Mloc_c sigma_c + Dloc_c^T p_c ; r_p,c = Dloc_c sigma_c - b_p,c.
__global__ void k_coarse_cell(LevelDev L, const double* __restrict__ sig, const double* __restrict__ p,
                              const double* __restrict__ bp, double* __restrict__ yl, double* __restrict__ rp,
                              double* __restrict__ kapc, int kind, double a, Reduce red) {
  double acc[1] = {0.0};
  GRID_STRIDE(c, L.nc) {
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c];
    const double* pc = p + po;
    double pb = 0.0;
    for (int r = 0; r < mc; ++r) pb = fma(L.w[po + r], pc[r], pb);
    const double kp = kappa_of(pb, kind, a);
    const double s = 1.0 / kp;
    if (kapc) kapc[c] = kp;
    double sl[kMaxLoc];
    for (int t = 0; t < nl; ++t) sl[t] = sig[L.loc[lo + t]];
    const double* M = L.Mloc + L.mat_off[c];
    const double* D = L.Dloc + L.dmat_off[c];
    for (int u = 0; u < nl; ++u) {
      double y = 0.0;
      for (int t = 0; t < nl; ++t) y = fma(M[u * nl + t], sl[t], y);
      y *= s;
      for (int r = 0; r < mc; ++r) y = fma(D[r * nl + u], pc[r], y);
      yl[lo + u] = y;
    }
    for (int r = 0; r < mc; ++r) {
      double v = 0.0;
      for (int t = 0; t < nl; ++t) v = fma(D[r * nl + t], sl[t], v);
      if (bp) v -= bp[po + r];
      rp[po + r] = v;
      acc[0] = fma(v, v, acc[0]);
    }
  }
  grid_reduce<1, false>(acc, red);
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

// Hybridization (Sec. 3.4): local saddles [s M D^T; D 0] with s = 1/kappa_c have the inverse
// [kappa A, B; B^T, C / kappa] where [A B; B^T C] is the stored kappa = 1 inverse.
// Right-hand side of H lambda = xi: per cell u = kappa A bhat + B b_p, scattered with the interface signs.
__global__ void k_hyb_rhs(LevelDev L, const double* __restrict__ kapc, const double* __restrict__ bs,
                          const double* __restrict__ bp, double* __restrict__ ylam) {
  GRID_STRIDE(c, L.nc) {
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const double kp = kapc[c];
    const double* S = L.Sinv + L.sad_off[c];
    double bh[kMaxLoc];
    for (int t = 0; t < nl; ++t) bh[t] = L.own0[lo + t] ? bs[L.loc[lo + t]] : 0.0;
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k) {
      const int u = L.if_slot[k];
      double a1 = 0.0, a2 = 0.0;
      for (int t = 0; t < nl; ++t) a1 = fma(S[u * n + t], bh[t], a1);
      for (int r = 0; r < mc; ++r) a2 = fma(S[u * n + nl + r], bp[po + r], a2);
      ylam[k] = L.if_sign[k] * fma(kp, a1, a2);
    }
  }
}

__global__ void k_lam_gather(LevelDev L, const double* __restrict__ ylam, double* __restrict__ out, int invert) {
  GRID_STRIDE(l, L.nlam) {
    double v = ylam[L.lam_y0[l]] + ylam[L.lam_y1[l]];
    out[l] = invert ? 1.0 / v : v;
  }
}

__global__ void k_hyb_diag_cells(LevelDev L, const double* __restrict__ kapc, double* __restrict__ ylam) {
  GRID_STRIDE(c, L.nc) {
    const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
    const double* H = L.Hc + L.hc_off[c];
    for (int k = 0; k < ni; ++k) ylam[k0 + k] = kapc[c] * H[k * ni + k];
  }
}

// per cell: ylam[k] = kappa_c sum_j Hc[k, j] pnew_j, with pnew = z + beta pold formed on the fly
__global__ void k_hyb_apply_cells(LevelDev L, const double* __restrict__ kapc, const double* __restrict__ z,
                                  const double* __restrict__ pold, const double* sc, int first,
                                  double* __restrict__ ylam) {
  const double beta = first ? 0.0 : sc[S_BETA];
  GRID_STRIDE(c, L.nc) {
    const int k0 = L.if_off[c], ni = L.if_off[c + 1] - k0;
    const double* H = L.Hc + L.hc_off[c];
    double v[kMaxLoc];
    for (int j = 0; j < ni; ++j) {
      const int l = L.if_lam[k0 + j];
      v[j] = first ? z[l] : fma(beta, pold[l], z[l]);
    }
    const double kp = kapc[c];
    for (int k = 0; k < ni; ++k) {
      double y = 0.0;
      for (int j = 0; j < ni; ++j) y = fma(H[k * ni + j], v[j], y);
      ylam[k0 + k] = kp * y;
    }
  }
}

__global__ void k_hyb_gather_dot(LevelDev L, const double* __restrict__ ylam, const double* __restrict__ z,
                                 const double* __restrict__ pold, double* __restrict__ pnew, double* __restrict__ q,
                                 double* sc, int first, Reduce red) {
  const double beta = first ? 0.0 : sc[S_BETA];
  double acc[1] = {0.0};
  GRID_STRIDE(l, L.nlam) {
    const double pl = first ? z[l] : fma(beta, pold[l], z[l]);
    const double y = ylam[L.lam_y0[l]] + ylam[L.lam_y1[l]];
    pnew[l] = pl;
    q[l] = y;
    acc[0] = fma(pl, y, acc[0]);
  }
  if (grid_reduce<1, false>(acc, red) && threadIdx.x == 0) {
    sc[S_PQ] = acc[0];
    sc[S_ALPHA] = acc[0] != 0.0 ? sc[S_RZ] / acc[0] : 0.0;
  }
}

// sigma^c = kappa A w + B b_p, p_c = B^T w + C b_p / kappa with w = bhat - C^T lambda
__global__ void k_hyb_recover(LevelDev L, const double* __restrict__ kapc, const double* __restrict__ bs,
                              const double* __restrict__ bp, const double* __restrict__ lam,
                              double* __restrict__ dsig, double* __restrict__ dp) {
  GRID_STRIDE(c, L.nc) {
    const int mc = L.m[c], lo = L.loc_off[c], nl = L.loc_off[c + 1] - lo, po = L.p_off[c], n = nl + mc;
    const double kp = kapc[c];
    const double* S = L.Sinv + L.sad_off[c];
    double w[kMaxLoc];
    for (int t = 0; t < nl; ++t) w[t] = L.own0[lo + t] ? bs[L.loc[lo + t]] : 0.0;
    for (int k = L.if_off[c]; k < L.if_off[c + 1]; ++k) w[L.if_slot[k]] -= L.if_sign[k] * lam[L.if_lam[k]];
    for (int u = 0; u < nl; ++u) {
      if (!L.own0[lo + u]) continue;
      double a1 = 0.0, a2 = 0.0;
      for (int t = 0; t < nl; ++t) a1 = fma(S[u * n + t], w[t], a1);
      for (int r = 0; r < mc; ++r) a2 = fma(S[u * n + nl + r], bp[po + r], a2);
      dsig[L.loc[lo + u]] = fma(kp, a1, a2);
    }
    for (int r = 0; r < mc; ++r) {
      double a1 = 0.0, a2 = 0.0;
      for (int t = 0; t < nl; ++t) a1 = fma(S[(nl + r) * n + t], w[t], a1);
      for (int q = 0; q < mc; ++q) a2 = fma(S[(nl + r) * n + nl + q], bp[po + q], a2);
      dp[po + r] = a1 + a2 / kp;
    }
  }
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------------------------------------

static std::atomic<long long> g_launches(0);
long long launch_count() { return g_launches.load(); }
#define COUNT(n) g_launches.fetch_add(n)

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
                     double* jdiag, Reduce red) {
  COUNT(1);
  k_residual<<<grid_for(F.N), kThreads, 0, st>>>(F, q, kap, dkap, g, rhs, R, Tval, dinv, diagT, jdiag, red);
}
void launch_jacobi_update(cudaStream_t st, int n, const double* q, const double* R, const double* jdiag,
                          const double* diagT, double omega, double* qnew) {
  COUNT(1);
  k_jacobi_update<<<grid_for(n), kThreads, 0, st>>>(n, q, R, jdiag, diagT, omega, qnew);
}
void launch_fine_spmv(cudaStream_t st, const FineDev& F, const double* Tval, const double* diagT, const double* z,
                      const double* pold, double* pnew, double* q, double* sc, int first, Reduce red) {
  COUNT(1);
  k_fine_spmv<<<grid_for(F.N), kThreads, 0, st>>>(F, Tval, diagT, z, pold, pnew, q, sc, first, red);
}
void launch_pcg_init(cudaStream_t st, int n, const double* b, double bscale, const double* dinv, double* x,
                     double* r, double* z, double* sc, Reduce red) {
  COUNT(1);
  k_pcg_init<<<grid_for(n), kThreads, 0, st>>>(n, b, bscale, dinv, x, r, z, sc, red);
}
void launch_pcg_update(cudaStream_t st, int n, double* x, double* r, double* z, const double* p, const double* q,
                       const double* dinv, double* sc, Reduce red) {
  COUNT(1);
  k_pcg_update<<<grid_for(n), kThreads, 0, st>>>(n, x, r, z, p, q, dinv, sc, red);
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
  k_csr<<<grid_for(nrows), kThreads, 0, st>>>(nrows, off, col, val, x, y, alpha, beta);
}
void launch_coarse_cell(cudaStream_t st, const LevelDev& L, const double* sig, const double* p, const double* bp,
                        double* yl, double* rp, double* kapc, int kind, double a, Reduce red) {
  COUNT(1);
  k_coarse_cell<<<grid_for(L.nc), kThreads, 0, st>>>(L, sig, p, bp, yl, rp, kapc, kind, a, red);
}
void launch_coarse_flux(cudaStream_t st, const LevelDev& L, const double* yl, const double* bs, double* rs,
                        Reduce red) {
  COUNT(1);
  k_coarse_flux<<<grid_for(L.nflux), kThreads, 0, st>>>(L, yl, bs, rs, red);
}
void launch_coarse_pbar_max(cudaStream_t st, const LevelDev& L, const double* dp, Reduce red) {
  COUNT(1);
  k_coarse_pbar_max<<<grid_for(L.nc), kThreads, 0, st>>>(L, dp, red);
}
void launch_hyb_rhs(cudaStream_t st, const LevelDev& L, const double* kapc, const double* bs, const double* bp,
                    double* ylam, double* xi) {
  COUNT(2);
  k_hyb_rhs<<<grid_for(L.nc), kThreads, 0, st>>>(L, kapc, bs, bp, ylam);
  k_lam_gather<<<grid_for(L.nlam), kThreads, 0, st>>>(L, ylam, xi, 0);
}
void launch_hyb_diag(cudaStream_t st, const LevelDev& L, const double* kapc, double* ylam, double* dinv) {
  COUNT(2);
  k_hyb_diag_cells<<<grid_for(L.nc), kThreads, 0, st>>>(L, kapc, ylam);
  k_lam_gather<<<grid_for(L.nlam), kThreads, 0, st>>>(L, ylam, dinv, 1);
}
void launch_hyb_spmv(cudaStream_t st, const LevelDev& L, const double* kapc, const double* z, const double* pold,
                     double* pnew, double* q, double* ylam, double* sc, int first, Reduce red) {
  COUNT(2);
  k_hyb_apply_cells<<<grid_for(L.nc), kThreads, 0, st>>>(L, kapc, z, pold, sc, first, ylam);
  k_hyb_gather_dot<<<grid_for(L.nlam), kThreads, 0, st>>>(L, ylam, z, pold, pnew, q, sc, first, red);
}
void launch_hyb_recover(cudaStream_t st, const LevelDev& L, const double* kapc, const double* bs, const double* bp,
                        const double* lam, double* dsig, double* dp) {
  COUNT(1);
  k_hyb_recover<<<grid_for(L.nc), kThreads, 0, st>>>(L, kapc, bs, bp, lam, dsig, dp);
}

}  // namespace nlmg
