// Small dense FP64 linear algebra used by the host-side hierarchy setup (row-major storage).
#pragma once
#include <vector>

namespace nlmg {

// Eigenpairs of the `k` smallest eigenvalues of the symmetric n x n matrix A (row-major, destroyed).
// Householder reduction to tridiagonal form, Sturm-sequence bisection for the eigenvalues, inverse iteration on
// the tridiagonal matrix with modified Gram-Schmidt inside clusters, then back-transformation.
// vals[k] ascending; vecs is n x k row-major (column j = eigenvector j, unit 2-norm).
void sym_eig_smallest(int n, std::vector<double>& A, int k, std::vector<double>& vals, std::vector<double>& vecs,
                      double* next_val = nullptr);

// One-sided Jacobi SVD of the n x m matrix V (row-major, m small): on return the columns of U (n x m) are the
// left singular vectors sorted by descending singular value s[m]. Columns with zero singular value are zero.
void jacobi_svd(int n, int m, const std::vector<double>& V, std::vector<double>& U, std::vector<double>& s);

// LU factorisation with partial pivoting of the n x n matrix A (in place); piv[n]. Returns false if singular.
bool lu_factor(int n, double* A, int* piv);
void lu_solve(int n, const double* LU, const int* piv, double* b);           // one right-hand side, in place
bool invert(int n, const double* A, double* Ainv);                            // Ainv = A^-1 via LU

// Cholesky A = L L^T of an SPD matrix (lower triangle written in place). Returns false if not SPD.
bool chol_factor(int n, double* A);
void chol_solve(int n, const double* L, double* b);
bool chol_upper_factor(int n, double* A);                         // A = U^T U on the upper triangle
void chol_upper_solve(int n, const double* U, double* b);
void chol_solve_multi(int n, const double* L, int nr, double* X);   // n x nr right-hand sides, row-major

}  // namespace nlmg
