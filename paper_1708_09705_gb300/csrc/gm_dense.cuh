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

namespace gmpic {

// Sub-catalogue lists (host): blk[k] = block of star k.  boff[nb + 1]: first
// row of each block in block order; coff[nb + 1]: offset of each block's
// N_k x N_k matrix; bidx[n]: star of each block-order row (stars of a block
// in increasing index); rowpos[n]: block-order row of each star; dims[nb]:
// N_k.  False when a block holds more than max_block stars.
inline bool block_lists(int64_t n, const int32_t* blk, int nb, int max_block, int64_t* boff,
                        int64_t* coff, int64_t* bidx, int32_t* rowpos, int32_t* dims) {
  for (int k = 0; k <= nb; ++k) boff[k] = coff[k] = 0;
  for (int64_t k = 0; k < n; ++k) boff[blk[k] + 1]++;
  for (int k = 0; k < nb; ++k) {
    dims[k] = (int32_t)boff[k + 1];
    if (dims[k] > max_block) return false;
    boff[k + 1] += boff[k];
    coff[k + 1] = coff[k] + (int64_t)dims[k] * dims[k];
  }
  for (int k = 0; k < nb; ++k) dims[k] = 0;  // fill counters
  for (int64_t k = 0; k < n; ++k) {
    const int b = blk[k];
    const int64_t r = boff[b] + dims[b]++;
    bidx[r] = k;
    rowpos[k] = (int32_t)r;
  }
  return true;
}

// Pair (a, b), a >= b, of the p-th lower-triangle entry in row-major order.
GM_HD inline void tri_index(int64_t p, int* a, int* b) {
  int64_t r = (int64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while (r * (r + 1) / 2 > p) --r;
  while ((r + 1) * (r + 2) / 2 <= p) ++r;
  *a = (int)r;
  *b = (int)(p - r * (r + 1) / 2);
}

// Quadrature inputs of inducing pair p: distances and chord |u_a - u_b|.
GM_HD inline void upair(int64_t p, const double* us, const double* ux, const double* uy,
                        const double* uz, double* si, double* sj, double* ch) {
  int a, b;
  tri_index(p, &a, &b);
  const double dx = ux[a] - ux[b], dy = uy[a] - uy[b], dz = uz[a] - uz[b];
  si[p] = us[a];
  sj[p] = us[b];
  ch[p] = sqrt(dx * dx + dy * dy + dz * dz);
}

// Taper of the covariance at 3-D separation d (Wendland: taper 0, hard
// cutoff: 1); zero beyond the cutoff.
GM_HD inline double taper_weight(double d, double inv_cut, int taper) {
  const double h = d * inv_cut;
  if (taper == 0) {
    const double u = 1.0 - h;
    return h < 1.0 ? u * u * u * u * (4.0 * h + 1.0) : 0.0;
  }
  return h <= 1.0 ? 1.0 : 0.0;
}

// K_uu[a][b] (lower) from the pair's untapered value kp[p], tapered by the
// 3-D separation as K is (Wendland: taper 0, hard cutoff: 1), and the prior
// mean at inducing point a when a == b (lognormal: form 0, first order: 1).
GM_HD inline void kuu_entry(int64_t p, int R, double inv_cut, int taper, int form,
                            double log_rho_bar, double sigma2, const double* us, const double* ch,
                            const double* kp, double* Kuu, double* mu_u) {
  int a, b;
  tri_index(p, &a, &b);
  const double sa = us[a], sb = us[b], ds = sa - sb;
  const double d = sqrt(ds * ds + sa * sb * ch[p] * ch[p]);
  const double v = a == b ? kp[p] : taper_weight(d, inv_cut, taper) * kp[p];
  Kuu[(int64_t)a * R + b] = v;
  if (a == b) mu_u[a] = log_rho_bar + log(sa) - (form == 0 ? 0.5 * v : 0.5 * sigma2);
}

// Entry e of the inducing points' CSR over the stars (row = inducing point,
// column = internal star) into row rowpos[star] of K_ku (block order).
GM_HD inline void kku_entry(int64_t e, int R, const int64_t* qptr, const int32_t* qcol,
                            const double* qval, const int32_t* rowpos, double* Kku) {
  int64_t lo = 0, hi = R;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (qptr[mid] <= e) lo = mid; else hi = mid;
  }
  Kku[(int64_t)rowpos[qcol[e]] * R + lo] = qval[e];
}

// Stored K_ij (0 when the pair is beyond the cutoff); columns sorted per row.
GM_HD inline double csr_entry(const int64_t* row_ptr, const int32_t* col, const double* val,
                              int64_t i, int32_t j) {
  int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < row_ptr[i + 1] && col[lo] == j) ? val[lo] : 0.0;
}

// Entry e of the concatenated blocks' C_k (lower triangles only).
GM_HD inline void cmat_entry(int64_t e, int nb, const int64_t* coff, const int64_t* boff, int R,
                             const int64_t* bidx, const int64_t* row_ptr, const int32_t* col,
                             const double* val, const double* A, const double* Kku,
                             const double* sig, double* C) {
  int lo = 0, hi = nb;  // block k: coff[k] <= e < coff[k + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (coff[mid] <= e) lo = mid; else hi = mid;
  }
  const int k = lo;
  const int64_t N = boff[k + 1] - boff[k];
  const int64_t loc = e - coff[k];
  const int64_t a = loc / N, b = loc - a * N;
  if (b > a) return;
  const int64_t ra = boff[k] + a, rb = boff[k] + b;
  const int64_t ia = bidx[ra], ib = bidx[rb];
  const double kab = csr_entry(row_ptr, col, val, ia, (int32_t)ib);
  C[e] = gmdense::c_entry(kab, A + ra * R, Kku + rb * R, R, a == b, sig[ia] * sig[ia]);
}

// Task t of the forward solves: block t / (R + 1), column t % (R + 1) (the
// last column is the right-hand side y).
GM_HD inline void fsolve_task(int64_t t, int R, const int64_t* coff, const int64_t* boff,
                              const double* C, double* X, double* yv) {
  const int k = (int)(t / (R + 1));
  const int c = (int)(t - (int64_t)k * (R + 1));
  const int N = (int)(boff[k + 1] - boff[k]);
  if (N == 0) return;
  const double* L = C + coff[k];
  if (c < R) gmdense::solve_lower(L, N, N, X + boff[k] * R + c, R);
  else gmdense::solve_lower(L, N, N, yv + boff[k], 1);
}

// Task e < R^2: Lambda (lower); e >= R^2: eta.
GM_HD inline void lambda_task(int64_t e, int64_t n, int R, const double* X, const double* yv,
                              double* Lam, double* eta) {
  if (e < (int64_t)R * R) {
    const int r1 = (int)(e / R), r2 = (int)(e - (int64_t)r1 * R);
    if (r2 <= r1) Lam[e] = gmdense::lambda_entry(X, n, R, r1, r2);
  } else {
    const int r = (int)(e - (int64_t)R * R);
    eta[r] = gmdense::eta_entry(X, yv, n, R, r);
  }
}

// Task e < R^2: P = K_uu^-1 + Lambda (lower); e >= R^2: h = K_uu^-1 mu_u + eta.
GM_HD inline void prec_task(int64_t e, int R, const double* Kinv, const double* Lam,
                            const double* mu_u, const double* eta, double* P, double* h) {
  if (e < (int64_t)R * R) {
    const int r1 = (int)(e / R), r2 = (int)(e - (int64_t)r1 * R);
    if (r2 <= r1) P[e] = Kinv[e] + Lam[e];
  } else {
    const int r = (int)(e - (int64_t)R * R);
    double v = eta[r];
    for (int c = 0; c < R; ++c) v += Kinv[(int64_t)r * R + c] * mu_u[c];
    h[r] = v;
  }
}

// Quadrature inputs of query-inducing pair p = q R + r.
GM_HD inline void qpair(int64_t p, int R, const double* qs, const double* qx, const double* qy,
                        const double* qz, const double* us, const double* ux, const double* uy,
                        const double* uz, double* si, double* sj, double* ch) {
  const int64_t q = p / R;
  const int r = (int)(p - q * R);
  const double dx = qx[q] - ux[r], dy = qy[q] - uy[r], dz = qz[q] - uz[r];
  si[p] = qs[q];
  sj[p] = us[r];
  ch[p] = sqrt(dx * dx + dy * dy + dz * dz);
}

// K_su[p] (p = q R + r) from the pair's untapered value, tapered as K.
GM_HD inline double ksu_entry(int64_t p, double inv_cut, int taper, const double* si,
                              const double* sj, const double* ch, const double* kp) {
  const double ds = si[p] - sj[p];
  const double d = sqrt(ds * ds + si[p] * sj[p] * ch[p] * ch[p]);
  return taper_weight(d, inv_cut, taper) * kp[p];
}

// Stored entry of star j in a query's CSR row [b, e) (columns sorted).
GM_HD inline double row_entry(const int32_t* col, const double* val, int64_t b, int64_t e,
                              int64_t j) {
  int64_t lo = b, hi = e;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < e && col[lo] == j) ? val[lo] : 0.0;
}

// PIC predictive of ln A at one query point assigned to block k (the
// paper's partially independent conditional, Sect. 4.1 / App. B): with
// A_s = k_su K_uu^-1, D = k_sk - K_ku A_s^T (the query's covariance with the
// block's observations given u), g = C_k^-1 D and L = A_s - g^T A_k,
//   mean = m_s + g^T (a~_k - m_k) + L (mean_u - mu_u),
//   var  = k_ss - A_s k_us - g^T D + L cov_u L^T.
// Lu, Ck: factors of K_uu and C_k; A, Kku: n x R in block order; ksu: R
// tapered cross-covariances; [qb, qe) the query's row of its CSR over the
// stars (tapered).  Scratch: As, Lc, t (R), D, g (N_k).
GM_HD inline void pic_point(int R, int k, const int64_t* boff, const int64_t* coff,
                            const int64_t* bidx, const double* Lu, const double* Cf,
                            const double* A, const double* Kku, const double* mu_u,
                            const double* pmean, const double* pcov, const double* obs,
                            const double* prior_m, const double* ksu, double kss, double ms,
                            int64_t qb, int64_t qe, const int32_t* qcol, const double* qval,
                            double* As, double* Lc, double* t, double* D, double* g,
                            double* mean, double* var) {
  const int64_t b0 = boff[k];
  const int N = (int)(boff[k + 1] - b0);
  for (int r = 0; r < R; ++r) As[r] = ksu[r];
  gmdense::solve_lower(Lu, R, R, As, 1);
  gmdense::solve_lower_t(Lu, R, R, As, 1);
  for (int a = 0; a < N; ++a) {
    const int64_t j = bidx[b0 + a];
    double v = row_entry(qcol, qval, qb, qe, j);
    const double* kr = Kku + (b0 + a) * R;
    for (int r = 0; r < R; ++r) v -= kr[r] * As[r];
    D[a] = v;
    g[a] = v;
  }
  if (N > 0) {
    gmdense::solve_lower(Cf + coff[k], N, N, g, 1);
    gmdense::solve_lower_t(Cf + coff[k], N, N, g, 1);
  }
  for (int r = 0; r < R; ++r) {
    double v = As[r];
    for (int a = 0; a < N; ++a) v -= g[a] * A[(b0 + a) * R + r];
    Lc[r] = v;
  }
  double m = ms, v = kss;
  for (int a = 0; a < N; ++a) {
    const int64_t j = bidx[b0 + a];
    m += g[a] * (obs[j] - prior_m[j]);
    v -= g[a] * D[a];
  }
  for (int r = 0; r < R; ++r) {
    m += Lc[r] * (pmean[r] - mu_u[r]);
    v -= As[r] * ksu[r];
    double tr = 0.0;
    for (int c = 0; c < R; ++c) tr += pcov[(int64_t)r * R + c] * Lc[c];
    t[r] = tr;
  }
  for (int r = 0; r < R; ++r) v += Lc[r] * t[r];
  *mean = m;
  *var = v;
}

}  // namespace gmpic
