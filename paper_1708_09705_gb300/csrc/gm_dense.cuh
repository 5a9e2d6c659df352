// Dense FP64 linear algebra of the PITC / PIC posterior over inducing points
// (Sect. 4.1, simplified case; the conditional of each sub-catalogue given
// the inducing values, App. B), written as per-output routines so that a
// device kernel runs them one thread per output (or, for the Cholesky
// factorisation, one thread block per matrix in barrier-separated phases)
// and a host build runs the same routines in the same order.
//
// Matrices are row-major with leading dimension ld; only lower triangles of
// symmetric matrices are read.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define GM_HD __host__ __device__
#else
#define GM_HD
#endif

namespace gmdense {

// ---------------------------------------------------------------- Cholesky
// Right-looking A = L L^T on the lower triangle, column j in three phases
// with a barrier after each: chol_diag (one thread), chol_col and
// chol_update (all threads, rows striped by tid).
GM_HD inline double chol_diag(double* A, int64_t ld, int j) {
  double d = A[(int64_t)j * ld + j];
  if (!(d > 0.0)) return -1.0;
  d = sqrt(d);
  A[(int64_t)j * ld + j] = d;
  return d;
}

GM_HD inline void chol_col(double* A, int64_t ld, int n, int j, double d, int tid, int nt) {
  for (int i = j + 1 + tid; i < n; i += nt) A[(int64_t)i * ld + j] /= d;
}

GM_HD inline void chol_update(double* A, int64_t ld, int n, int j, int tid, int nt) {
  for (int i = j + 1 + tid; i < n; i += nt) {
    const double aij = A[(int64_t)i * ld + j];
    double* Ai = A + (int64_t)i * ld;
    for (int k = j + 1; k <= i; ++k) Ai[k] -= aij * A[(int64_t)k * ld + j];
  }
}

// ---------------------------------------------------------------- solves
// L x = b in place (x strided by inc).
GM_HD inline void solve_lower(const double* L, int64_t ld, int n, double* x, int64_t inc) {
  for (int i = 0; i < n; ++i) {
    double v = x[(int64_t)i * inc];
    const double* Li = L + (int64_t)i * ld;
    for (int k = 0; k < i; ++k) v -= Li[k] * x[(int64_t)k * inc];
    x[(int64_t)i * inc] = v / Li[i];
  }
}

// L^T x = b in place.
GM_HD inline void solve_lower_t(const double* L, int64_t ld, int n, double* x, int64_t inc) {
  for (int i = n - 1; i >= 0; --i) {
    double v = x[(int64_t)i * inc];
    for (int k = i + 1; k < n; ++k) v -= L[(int64_t)k * ld + i] * x[(int64_t)k * inc];
    x[(int64_t)i * inc] = v / L[(int64_t)i * ld + i];
  }
}

// ---------------------------------------------------------------- PITC steps
// Row j of A = K_ku K_uu^-1 (R values): a = K_uu^-1 k with k the star's row
// of K_ku; Lu = chol(K_uu).
GM_HD inline void a_row(const double* Lu, int R, const double* kku_row, double* a_row_out) {
  for (int r = 0; r < R; ++r) a_row_out[r] = kku_row[r];
  solve_lower(Lu, R, R, a_row_out, 1);
  solve_lower_t(Lu, R, R, a_row_out, 1);
}

// Entry (a, b), b <= a, of the block's noisy conditional covariance
// C = K_kk - A K_uk + diag(sigma^2): kab = K_kk[a][b].
GM_HD inline double c_entry(double kab, const double* A_a, const double* Kku_b, int R, bool diag,
                            double sig2_a) {
  double v = kab;
  for (int r = 0; r < R; ++r) v -= A_a[r] * Kku_b[r];
  return diag ? v + sig2_a : v;
}

// Entry a of y = atil - m + A mu_u: with p(atil_k | u) =
// N(m_k + A_k (u - mu_u), C_k) the block's factor in u is
// exp(-u^T Lambda_k u / 2 + eta_k^T u) with Lambda_k = A_k^T C_k^-1 A_k and
// eta_k = A_k^T C_k^-1 y_k.
GM_HD inline double y_entry(double atil_a, double m_a, const double* A_a, const double* mu_u,
                            int R) {
  double v = atil_a - m_a;
  for (int r = 0; r < R; ++r) v += A_a[r] * mu_u[r];
  return v;
}

// Lambda[r1][r2] = sum_j X[j][r1] X[j][r2] over all n stars (X: n x R).
GM_HD inline double lambda_entry(const double* X, int64_t n, int R, int r1, int r2) {
  double v = 0.0;
  for (int64_t j = 0; j < n; ++j) v += X[j * R + r1] * X[j * R + r2];
  return v;
}

// eta[r] = sum_j X[j][r] yv[j].
GM_HD inline double eta_entry(const double* X, const double* yv, int64_t n, int R, int r) {
  double v = 0.0;
  for (int64_t j = 0; j < n; ++j) v += X[j * R + r] * yv[j];
  return v;
}

// Column c of (L L^T)^-1 into col (R values, strided by inc).
GM_HD inline void inverse_col(const double* L, int R, int c, double* col, int64_t inc) {
  for (int r = 0; r < R; ++r) col[(int64_t)r * inc] = r == c ? 1.0 : 0.0;
  solve_lower(L, R, R, col, inc);
  solve_lower_t(L, R, R, col, inc);
}

}  // namespace gmdense
