// Small dense FP64 linear algebra for the host-side setup. Written from the textbook algorithms named at each
// routine (Householder tridiagonalisation, Sturm bisection, inverse iteration, Hestenes one-sided Jacobi SVD,
// LU with partial pivoting, Cholesky).
#include "dense.hpp"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>

namespace nlmg {

namespace {

// Number of eigenvalues of the symmetric tridiagonal (d, e) strictly below x (Sturm sequence / LDL^T inertia).
int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (std::fabs(q) < pivmin) q = -pivmin;
  if (q < 0) cnt++;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (std::fabs(q) < pivmin) q = -pivmin;
    if (q < 0) cnt++;
  }
  return cnt;
}

// Solve (T - lam I) x = b for the tridiagonal T = (d, e) by Gaussian elimination with partial pivoting.
void tri_shift_solve(int n, const double* d, const double* e, double lam, double tiny, double* b,
                     std::vector<double>& a0, std::vector<double>& a1, std::vector<double>& a2,
                     std::vector<double>& low) {
  // row i after elimination: a0[i] x_i + a1[i] x_{i+1} + a2[i] x_{i+2} = b_i
  a0.assign(n, 0.0);
  a1.assign(n, 0.0);
  a2.assign(n, 0.0);
  low.assign(n, 0.0);
  // current pending row (diag, super) and next row (sub, diag, super)
  double cd = d[0] - lam, cs = (n > 1) ? e[0] : 0.0, css = 0.0;
  for (int i = 0; i < n - 1; ++i) {
    double sub = e[i], nd = d[i + 1] - lam, ns = (i + 2 < n) ? e[i + 1] : 0.0;
    if (std::fabs(sub) > std::fabs(cd)) {
      // swap rows i and i+1
      double m = cd / sub;
      a0[i] = sub;
      a1[i] = nd;
      a2[i] = ns;
      std::swap(b[i], b[i + 1]);
      b[i + 1] -= m * b[i];
      double ncd = cs - m * nd, ncs = css - m * ns;
      cd = ncd;
      cs = ncs;
      css = 0.0;
    } else {
      if (cd == 0.0) cd = tiny;
      double m = sub / cd;
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
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    if (i + 1 < n) s -= a1[i] * b[i + 1];
    if (i + 2 < n) s -= a2[i] * b[i + 2];
    double piv = a0[i];
    if (std::fabs(piv) < tiny) piv = (piv < 0 ? -tiny : tiny);
    b[i] = s / piv;
  }
}

}  // namespace

void sym_eig_smallest(int n, std::vector<double>& A, int k, std::vector<double>& vals, std::vector<double>& vecs,
                      double* next_val) {
  vals.assign(k, 0.0);
  vecs.assign((size_t)n * k, 0.0);
  if (n == 0 || k == 0) return;
  if (n == 1) {
    vals[0] = A[0];
    vecs[0] = 1.0;
    if (next_val) *next_val = std::numeric_limits<double>::infinity();
    return;
  }
  // --- Householder reduction: A = Q T Q^T, reflectors stored below the subdiagonal --------------------------
  std::vector<double> d(n), e(n, 0.0), beta(n, 0.0), v(n), p(n), w(n);
  for (int kk = 0; kk < n - 2; ++kk) {
    int m = n - kk - 1;  // length of x = A[kk+1:, kk]
    double* col = &v[0];
    double nrm2 = 0.0;
    for (int i = 0; i < m; ++i) {
      col[i] = A[(size_t)(kk + 1 + i) * n + kk];
      nrm2 += col[i] * col[i];
    }
    double alpha = std::sqrt(nrm2);
    if (alpha == 0.0) {
      beta[kk] = 0.0;
      e[kk] = 0.0;
      for (int i = 0; i < m; ++i) A[(size_t)(kk + 1 + i) * n + kk] = 0.0;
      continue;
    }
    if (col[0] > 0) alpha = -alpha;   // x -> alpha e1, v = x - alpha e1 (no cancellation)
    col[0] -= alpha;
    double vn2 = 0.0;
    for (int i = 0; i < m; ++i) vn2 += col[i] * col[i];
    double b = 2.0 / vn2;
    beta[kk] = b;
    e[kk] = alpha;
    // p = b * A22 v ; w = p - (b/2)(p.v) v ; A22 -= v w^T + w v^T
    for (int i = 0; i < m; ++i) {
      const double* Ai = &A[(size_t)(kk + 1 + i) * n + kk + 1];
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += Ai[j] * col[j];
      p[i] = b * s;
    }
    double pv = 0.0;
    for (int i = 0; i < m; ++i) pv += p[i] * col[i];
    for (int i = 0; i < m; ++i) w[i] = p[i] - 0.5 * b * pv * col[i];
    for (int i = 0; i < m; ++i) {
      double* Ai = &A[(size_t)(kk + 1 + i) * n + kk + 1];
      for (int j = 0; j < m; ++j) Ai[j] -= col[i] * w[j] + w[i] * col[j];
    }
    for (int i = 0; i < m; ++i) A[(size_t)(kk + 1 + i) * n + kk] = col[i];  // keep reflector
  }
  for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
  // reflector for column n-2 is absent: mark
  beta[n - 2] = 0.0;
  std::vector<double> e2(n, 0.0);
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(e[i]) : 0.0);
    tnorm = std::max(tnorm, r);
  }
  for (int i = 0; i < n - 1; ++i) e2[i] = e[i] * e[i];
  const double eps = std::numeric_limits<double>::epsilon();
  double pivmin = std::max(std::numeric_limits<double>::min(), eps * eps * tnorm * tnorm) + 1e-300;
  double glo = -tnorm, ghi = tnorm;
  int want = std::min(k + 1, n);
  std::vector<double> lam(want);
  for (int j = 0; j < want; ++j) {
    double lo = glo, hi = ghi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (sturm_count(n, d.data(), e2.data(), mid, pivmin) > j) hi = mid; else lo = mid;
      if (hi - lo <= 2.0 * eps * std::max(std::fabs(lo), std::fabs(hi)) + 1e-300) break;
    }
    lam[j] = 0.5 * (lo + hi);
  }
  if (next_val) *next_val = (want > k) ? lam[k] : std::numeric_limits<double>::infinity();
  // --- inverse iteration on T --------------------------------------------------------------------------------
  std::vector<double> Z((size_t)n * k, 0.0), x(n), a0, a1, a2, low;
  double tiny = eps * std::max(tnorm, 1e-300);
  double cluster_tol = 1e-3 * std::max(tnorm, 1e-300);
  int cstart = 0;
  for (int j = 0; j < k; ++j) {
    vals[j] = lam[j];
    if (j > 0 && std::fabs(lam[j] - lam[j - 1]) > cluster_tol) cstart = j;
    // deterministic start vector
    uint64_t s = 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1);
    for (int i = 0; i < n; ++i) {
      s ^= s << 13; s ^= s >> 7; s ^= s << 17;
      x[i] = ((double)(s >> 11) / 9007199254740992.0) - 0.5;
    }
    double shift = lam[j];
    for (int it = 0; it < 4; ++it) {
      tri_shift_solve(n, d.data(), e.data(), shift, tiny, x.data(), a0, a1, a2, low);
      for (int q = cstart; q < j; ++q) {  // orthogonalise inside the cluster
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += x[i] * Z[(size_t)i * k + q];
        for (int i = 0; i < n; ++i) x[i] -= dot * Z[(size_t)i * k + q];
      }
      double nr = 0.0;
      for (int i = 0; i < n; ++i) nr += x[i] * x[i];
      nr = std::sqrt(nr);
      if (nr == 0.0) { x.assign(n, 0.0); x[j % n] = 1.0; nr = 1.0; }
      for (int i = 0; i < n; ++i) x[i] /= nr;
    }
    for (int i = 0; i < n; ++i) Z[(size_t)i * k + j] = x[i];
  }
  // --- back-transformation y = H_0 H_1 ... H_{n-3} z -----------------------------------------------------------
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < n; ++i) x[i] = Z[(size_t)i * k + j];
    for (int kk = n - 3; kk >= 0; --kk) {
      if (beta[kk] == 0.0) continue;
      int m = n - kk - 1;
      double dot = 0.0;
      for (int i = 0; i < m; ++i) dot += A[(size_t)(kk + 1 + i) * n + kk] * x[kk + 1 + i];
      dot *= beta[kk];
      for (int i = 0; i < m; ++i) x[kk + 1 + i] -= dot * A[(size_t)(kk + 1 + i) * n + kk];
    }
    for (int i = 0; i < n; ++i) vecs[(size_t)i * k + j] = x[i];
  }
}

void jacobi_svd(int n, int m, const std::vector<double>& V, std::vector<double>& U, std::vector<double>& s) {
  U = V;
  s.assign(m, 0.0);
  const double eps = std::numeric_limits<double>::epsilon();
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) {
        double a = 0, b = 0, g = 0;
        for (int r = 0; r < n; ++r) {
          double ui = U[(size_t)r * m + i], uj = U[(size_t)r * m + j];
          a += ui * ui;
          b += uj * uj;
          g += ui * uj;
        }
        if (std::fabs(g) <= eps * std::sqrt(a * b) || g == 0.0) continue;
        rotated = true;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int r = 0; r < n; ++r) {
          double ui = U[(size_t)r * m + i], uj = U[(size_t)r * m + j];
          U[(size_t)r * m + i] = c * ui - sn * uj;
          U[(size_t)r * m + j] = sn * ui + c * uj;
        }
      }
    if (!rotated) break;
  }
  std::vector<int> order(m);
  std::vector<double> nrm(m);
  for (int j = 0; j < m; ++j) {
    double a = 0;
    for (int r = 0; r < n; ++r) a += U[(size_t)r * m + j] * U[(size_t)r * m + j];
    nrm[j] = std::sqrt(a);
    order[j] = j;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  std::vector<double> out((size_t)n * m, 0.0);
  for (int jj = 0; jj < m; ++jj) {
    int j = order[jj];
    s[jj] = nrm[j];
    if (nrm[j] > 0)
      for (int r = 0; r < n; ++r) out[(size_t)r * m + jj] = U[(size_t)r * m + j] / nrm[j];
  }
  U.swap(out);
}

bool lu_factor(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double mx = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > mx) { mx = std::fabs(A[(size_t)i * n + k]); p = i; }
    piv[k] = p;
    if (mx == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    double inv = 1.0 / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double f = A[(size_t)i * n + k] * inv;
      A[(size_t)i * n + k] = f;
      if (f != 0.0) {
        double* Ai = &A[(size_t)i * n];
        const double* Ak = &A[(size_t)k * n];
        for (int j = k + 1; j < n; ++j) Ai[j] -= f * Ak[j];
      }
    }
  }
  return true;
}

void lu_solve(int n, const double* LU, const int* piv, double* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 1; i < n; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s / LU[(size_t)i * n + i];
  }
}

bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> LU(A, A + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, LU.data(), piv.data())) return false;
  std::vector<double> col(n);
  for (int j = 0; j < n; ++j) {
    std::fill(col.begin(), col.end(), 0.0);
    col[j] = 1.0;
    lu_solve(n, LU.data(), piv.data(), col.data());
    for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + j] = col[i];
  }
  return true;
}

// Left-looking Cholesky, L in the lower triangle. Every entry is one dot product summed in k order; eight rows of a
// column are summed side by side (independent chains, each in the same order as alone), which hides the add latency
// without changing a single rounding.
bool chol_factor(int n, double* A) {
  for (int j = 0; j < n; ++j) {
    const double* Aj = A + (size_t)j * n;
    double s = Aj[j];
    for (int k = 0; k < j; ++k) s -= Aj[k] * Aj[k];
    if (!(s > 0.0)) return false;
    double ljj = std::sqrt(s);
    A[(size_t)j * n + j] = ljj;
    int i = j + 1;
    for (; i + 8 <= n; i += 8) {
      double* R[8];
      double t[8];
      for (int u = 0; u < 8; ++u) {
        R[u] = A + (size_t)(i + u) * n;
        t[u] = R[u][j];
      }
      for (int k = 0; k < j; ++k) {
        const double a = Aj[k];
        t[0] -= R[0][k] * a;
        t[1] -= R[1][k] * a;
        t[2] -= R[2][k] * a;
        t[3] -= R[3][k] * a;
        t[4] -= R[4][k] * a;
        t[5] -= R[5][k] * a;
        t[6] -= R[6][k] * a;
        t[7] -= R[7][k] * a;
      }
      for (int u = 0; u < 8; ++u) R[u][j] = t[u] / ljj;
    }
    for (; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * Aj[k];
      A[(size_t)i * n + j] = t / ljj;
    }
  }
  return true;
}

void chol_solve(int n, const double* L, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
}

// L L^T X = B for nr right-hand sides stored row-major (n x nr), in place; same operation order per entry as
// chol_solve (subtractions in k order, then the division). The right-hand sides are taken eight at a time with their
// running values in registers, so that a block of X stays in L1 and no entry is stored before it is final; the back
// substitution reads L^T by rows.
void chol_solve_multi(int n, const double* L, int nr, double* X) {
  constexpr int W = 8;
  std::vector<double> Lt((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < k; ++i) Lt[(size_t)i * n + k] = L[(size_t)k * n + i];
  for (int r0 = 0; r0 < nr; r0 += W) {
    const int w = std::min(W, nr - r0);
    if (w == W) {
      for (int i = 0; i < n; ++i) {
        double* Xi = X + (size_t)i * nr + r0;
        double a[W];
        for (int u = 0; u < W; ++u) a[u] = Xi[u];
        const double* Li = L + (size_t)i * n;
        for (int k = 0; k < i; ++k) {
          const double l = Li[k];
          if (l == 0.0) continue;
          const double* Xk = X + (size_t)k * nr + r0;
          for (int u = 0; u < W; ++u) a[u] -= l * Xk[u];
        }
        const double d = Li[i];
        for (int u = 0; u < W; ++u) Xi[u] = a[u] / d;
      }
      for (int i = n - 1; i >= 0; --i) {
        double* Xi = X + (size_t)i * nr + r0;
        double a[W];
        for (int u = 0; u < W; ++u) a[u] = Xi[u];
        const double* Ui = Lt.data() + (size_t)i * n;
        for (int k = i + 1; k < n; ++k) {
          const double l = Ui[k];
          if (l == 0.0) continue;
          const double* Xk = X + (size_t)k * nr + r0;
          for (int u = 0; u < W; ++u) a[u] -= l * Xk[u];
        }
        const double d = L[(size_t)i * n + i];
        for (int u = 0; u < W; ++u) Xi[u] = a[u] / d;
      }
    } else {
      for (int i = 0; i < n; ++i) {
        double* Xi = X + (size_t)i * nr + r0;
        const double* Li = L + (size_t)i * n;
        for (int k = 0; k < i; ++k) {
          const double l = Li[k];
          if (l == 0.0) continue;
          const double* Xk = X + (size_t)k * nr + r0;
          for (int u = 0; u < w; ++u) Xi[u] -= l * Xk[u];
        }
        const double d = Li[i];
        for (int u = 0; u < w; ++u) Xi[u] /= d;
      }
      for (int i = n - 1; i >= 0; --i) {
        double* Xi = X + (size_t)i * nr + r0;
        const double* Ui = Lt.data() + (size_t)i * n;
        for (int k = i + 1; k < n; ++k) {
          const double l = Ui[k];
          if (l == 0.0) continue;
          const double* Xk = X + (size_t)k * nr + r0;
          for (int u = 0; u < w; ++u) Xi[u] -= l * Xk[u];
        }
        const double d = L[(size_t)i * n + i];
        for (int u = 0; u < w; ++u) Xi[u] /= d;
      }
    }
  }
}

// Right-looking Cholesky on the upper triangle of a row-major SPD matrix: A = U^T U, U written over the upper
// triangle. Zero multipliers are skipped, so a sparse A (a cell-graph Laplacian in a banded order) costs in
// proportion to its fill rather than n^3.
bool chol_upper_factor(int n, double* A) {
  for (int k = 0; k < n; ++k) {
    double* Ak = A + (size_t)k * n;
    if (!(Ak[k] > 0.0)) return false;
    const double ukk = std::sqrt(Ak[k]);
    const double inv = 1.0 / ukk;
    Ak[k] = ukk;
    for (int j = k + 1; j < n; ++j) Ak[j] *= inv;
    for (int i = k + 1; i < n; ++i) {
      const double u = Ak[i];
      if (u == 0.0) continue;
      double* Ai = A + (size_t)i * n;
      for (int j = i; j < n; ++j) Ai[j] -= u * Ak[j];
    }
  }
  return true;
}

// U^T U x = b in place, U from chol_upper_factor.
void chol_upper_solve(int n, const double* U, double* b) {
  for (int k = 0; k < n; ++k) {
    const double* Uk = U + (size_t)k * n;
    const double y = b[k] / Uk[k];
    b[k] = y;
    if (y != 0.0)
      for (int j = k + 1; j < n; ++j) b[j] -= Uk[j] * y;
  }
  for (int i = n - 1; i >= 0; --i) {
    const double* Ui = U + (size_t)i * n;
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= Ui[j] * b[j];
    b[i] = s / Ui[i];
  }
}

}  // namespace nlmg
