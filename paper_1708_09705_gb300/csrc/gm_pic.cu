// PITC / PIC posterior of the log-extinction at inducing points (Sect. 4.1,
// the simplified case: hyperparameters fixed and each star's observed log-
// extinction Gaussian, a~_n | a_n ~ N(a_n, sigma_n^2)).
//
// The stars are split into sub-catalogues (blocks).  Given the values u at R
// inducing points the blocks are independent (PITC), each with the exact GP
// conditional a_k | u ~ N(m_k + A_k (u - mu_u), K_kk - A_k K_uk),
// A_k = K_ku K_uu^-1, so a~_k | u ~ N(m_k + A_k (u - mu_u), C_k) with
// C_k = K_kk - A_k K_uk + diag(sigma_k^2).  The block-site EP of the paper
// reaches its fixed point in one parallel sweep here (every factor is
// Gaussian), and the posterior of u is
//   P = K_uu^-1 + sum_k A_k^T C_k^-1 A_k,  h = K_uu^-1 mu_u + sum_k A_k^T C_k^-1 y_k,
//   y_k = a~_k - m_k + A_k mu_u,   mean = P^-1 h,   cov = P^-1.
// K_kk are read from the stored covariance, K_ku and K_uu come from the same
// sightline quadrature, cutoff and taper.  The dense algebra (FP64) is in
// gm_dense.cuh; here each step is a kernel with one thread per output, and the
// Cholesky factorisations run one thread block per matrix.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gm_dense.cuh"
#include "gm_internal.cuh"

namespace gm {

// Lower Cholesky factor in place of each dim[b] x dim[b] row-major matrix at
// base + off[b]; one thread block per matrix.
__global__ void __launch_bounds__(256) k_pic_chol(double* __restrict__ base,
                                                  const int64_t* __restrict__ off,
                                                  const int32_t* __restrict__ dim,
                                                  unsigned* __restrict__ flags) {
  __shared__ double d_s;
  __shared__ int bad;
  double* A = base + off[blockIdx.x];
  const int n = dim[blockIdx.x];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = gmdense::chol_diag(A, n, j);
      d_s = d;
      if (!(d > 0.0)) bad = 1;
    }
    __syncthreads();
    if (bad) break;
    gmdense::chol_col(A, n, n, j, d_s, threadIdx.x, blockDim.x);
    __syncthreads();
    gmdense::chol_update(A, n, n, j, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(flags, kFlagNotSPD);
}

// Quadrature inputs of the inducing pairs (a, b), a >= b, diagonal included.
__global__ void k_pic_upairs(int R, const double* __restrict__ us, const double* __restrict__ ux,
                             const double* __restrict__ uy, const double* __restrict__ uz,
                             double* __restrict__ si, double* __restrict__ sj,
                             double* __restrict__ ch) {
  const int64_t np = (int64_t)R * (R + 1) / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    gmpic::upair(p, us, ux, uy, uz, si, sj, ch);
  }
}

// K_uu (lower triangle, tapered as K) and the prior mean at the inducing
// points from the pairs' untapered values.
__global__ void k_pic_kuu(int R, double inv_cut, int taper, int form, double log_rho_bar,
                          double sigma2, const double* __restrict__ us,
                          const double* __restrict__ ch, const double* __restrict__ kp,
                          double* __restrict__ Kuu, double* __restrict__ mu_u) {
  const int64_t np = (int64_t)R * (R + 1) / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    gmpic::kuu_entry(p, R, inv_cut, taper == GM_TAPER_WENDLAND ? 0 : 1,
                     form == GM_FORM_LOGNORMAL ? 0 : 1, log_rho_bar, sigma2, us, ch, kp, Kuu,
                     mu_u);
  }
}

// K_ku rows in block order from the inducing points' CSR over the stars.
__global__ void k_pic_kku(int R, const int64_t* __restrict__ qptr,
                          const int32_t* __restrict__ qcol, const double* __restrict__ qval,
                          int64_t qnnz, const int32_t* __restrict__ rowpos,
                          double* __restrict__ Kku) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qnnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    gmpic::kku_entry(e, R, qptr, qcol, qval, rowpos, Kku);
  }
}

__global__ void k_pic_arow(int64_t n, int R, const double* __restrict__ Lu,
                           const double* __restrict__ Kku, double* __restrict__ A) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    gmdense::a_row(Lu, R, Kku + j * R, A + j * R);
}

// Lower triangle of every block's C_k = K_kk - A_k K_uk + diag(sigma^2).
__global__ void k_pic_cmat(int nb, const int64_t* __restrict__ coff,
                           const int64_t* __restrict__ boff, int R,
                           const int64_t* __restrict__ bidx, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ A, const double* __restrict__ Kku,
                           const double* __restrict__ sig, double* __restrict__ C) {
  const int64_t total = coff[nb];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    gmpic::cmat_entry(e, nb, coff, boff, R, bidx, row_ptr, col, val, A, Kku, sig, C);
  }
}

__global__ void k_pic_y(int64_t n, int R, const int64_t* __restrict__ bidx,
                        const double* __restrict__ obs, const double* __restrict__ prior_m,
                        const double* __restrict__ A, const double* __restrict__ mu_u,
                        double* __restrict__ yv) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    yv[j] = gmdense::y_entry(obs[bidx[j]], prior_m[bidx[j]], A + j * R, mu_u, R);
}

// X_k = L_k^-1 A_k (columns c < R) and yv_k = L_k^-1 y_k (c = R).
__global__ void k_pic_fsolve(int nb, int R, const int64_t* __restrict__ coff,
                             const int64_t* __restrict__ boff, const double* __restrict__ C,
                             double* __restrict__ X, double* __restrict__ yv) {
  const int64_t total = (int64_t)nb * (R + 1);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    gmpic::fsolve_task(t, R, coff, boff, C, X, yv);
  }
}

// Lambda (lower triangle) and eta over all stars.
__global__ void k_pic_lambda(int64_t n, int R, const double* __restrict__ X,
                             const double* __restrict__ yv, double* __restrict__ Lam,
                             double* __restrict__ eta) {
  const int64_t total = (int64_t)R * R + R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    gmpic::lambda_task(e, n, R, X, yv, Lam, eta);
  }
}

// Columns of (L L^T)^-1 (one thread per column).
__global__ void k_pic_inverse(int R, const double* __restrict__ L, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x)
    gmdense::inverse_col(L, R, c, out + c, R);
}

// P = K_uu^-1 + Lambda (lower triangle) and h = K_uu^-1 mu_u + eta.
__global__ void k_pic_prec(int R, const double* __restrict__ Kinv, const double* __restrict__ Lam,
                           const double* __restrict__ mu_u, const double* __restrict__ eta,
                           double* __restrict__ P, double* __restrict__ h) {
  const int64_t total = (int64_t)R * R + R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    gmpic::prec_task(e, R, Kinv, Lam, mu_u, eta, P, h);
  }
}

// mean = P^-1 h from the factor of P (one thread).
__global__ void k_pic_mean(int R, const double* __restrict__ LP, const double* __restrict__ h,
                           double* __restrict__ mean) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int r = 0; r < R; ++r) mean[r] = h[r];
  gmdense::solve_lower(LP, R, R, mean, 1);
  gmdense::solve_lower_t(LP, R, R, mean, 1);
}

static int grid_for(gm_ctx* c, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 128), 16 * sm_count(c)));
}

gm_status pic_posterior(gm_ctx* c, int R, const double* us, const double* ux, const double* uy,
                        const double* uz, const int32_t* h_block_int, int nb, double* mean,
                        double* cov) {
  const int64_t n = c->n;
  // ---- block lists (host): stars of block k in internal order
  std::vector<int64_t> boff(nb + 1), coff(nb + 1), bidx(n);
  std::vector<int32_t> rowpos(n), dims(nb);
  if (!gmpic::block_lists(n, h_block_int, nb, kMaxPicBlock, boff.data(), coff.data(), bidx.data(),
                          rowpos.data(), dims.data()))
    return set_error(c, GM_E_INVAL, "a sub-catalogue has more than 8192 stars");
  const int64_t RR = (int64_t)R * R;
  const int64_t npair = (int64_t)R * (R + 1) / 2;
  // device buffers
  ScopedDev b_i64(c, (size_t)(2 * (nb + 1) + n) * sizeof(int64_t));
  ScopedDev b_i32(c, (size_t)(n + nb + 1) * sizeof(int32_t));
  // Kuu, Lu, Kinv, Lam, P (R x R); mu_u, eta, h (R); pair inputs (4 npair);
  // Kku, A, X (n x R); yv (n); C (sum N_k^2)
  const size_t nd = 5 * RR + 3 * R + 4 * npair + 3 * n * (int64_t)R + n + coff[nb];
  ScopedDev b_d(c, std::max<size_t>(nd, 1) * sizeof(double));
  ScopedDev b_q(c, (size_t)(R + 1) * sizeof(int64_t));
  if (!b_i64.p || !b_i32.p || !b_d.p || !b_q.p) return set_error(c, GM_E_NOMEM, "PIC arrays");
  int64_t* d_boff = (int64_t*)b_i64.p;
  int64_t* d_coff = d_boff + nb + 1;
  int64_t* d_bidx = d_coff + nb + 1;
  int32_t* d_rowpos = (int32_t*)b_i32.p;
  int32_t* d_dims = d_rowpos + n;
  double* Kuu = (double*)b_d.p;
  double *Lu = Kuu + RR, *Kinv = Lu + RR, *Lam = Kinv + RR, *P = Lam + RR;
  double *mu_u = P + RR, *eta = mu_u + R, *h = eta + R;
  double *psi = h + R, *psj = psi + npair, *pch = psj + npair, *pk = pch + npair;
  double *Kku = pk + npair, *A = Kku + n * (int64_t)R, *X = A + n * (int64_t)R;
  double *yv = X + n * (int64_t)R, *C = yv + n;
  cudaStream_t st = c->stream;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_boff, boff.data(), (nb + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_coff, coff.data(), (nb + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_bidx, bidx.data(), n * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_rowpos, rowpos.data(), n * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_dims, dims.data(), nb * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemsetAsync(Kku, 0, n * (int64_t)R * sizeof(double), st));
  // ---- K_ku: the inducing points' neighbour CSR over the stars
  int64_t* qptr = (int64_t*)b_q.p;
  Buffer qcol;
  int64_t qnnz = 0;
  gm_status s = neighbour_csr(c, R, us, ux, uy, uz, nullptr, false, qptr, qcol, &qnnz, nullptr);
  if (s != GM_OK) return s;
  ScopedDev b_qv(c, (size_t)std::max<int64_t>(qnnz, 1) * sizeof(double));
  if (!b_qv.p) return set_error(c, GM_E_NOMEM, "PIC cross-covariances");
  s = pair_quadrature(c, R, us, ux, uy, uz, nullptr, qptr, (const int32_t*)qcol.p, qnnz, b_qv.p,
                      false);
  if (s != GM_OK) return s;
  if (qnnz > 0) {
    GM_PROF(c, "k_pic_kku");
    k_pic_kku<<<grid_for(c, qnnz), 128, 0, st>>>(R, qptr, (const int32_t*)qcol.p,
                                                 (const double*)b_qv.p, qnnz, d_rowpos, Kku);
    GM_LAUNCH_CHECK(c);
  }
  // ---- K_uu and the prior mean at the inducing points
  GM_PROF(c, "k_pic_upairs");
  k_pic_upairs<<<grid_for(c, npair), 128, 0, st>>>(R, us, ux, uy, uz, psi, psj, pch);
  GM_LAUNCH_CHECK(c);
  s = pairlist_quadrature(c, npair, psi, psj, pch, pk);
  if (s != GM_OK) return s;
  GM_PROF(c, "k_pic_kuu");
  k_pic_kuu<<<grid_for(c, npair), 128, 0, st>>>(R, 1.0 / c->cfg.cutoff_pc, c->cfg.taper,
                                                c->cfg.form, std::log(c->cfg.rho_bar),
                                                c->cfg.sigma2, us, pch, pk, Kuu, mu_u);
  GM_LAUNCH_CHECK(c);
  // ---- factor K_uu; A = K_ku K_uu^-1
  GM_CUDA_CHECK(c, cudaMemcpyAsync(Lu, Kuu, RR * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ScopedDev b_one(c, sizeof(int64_t) + sizeof(int32_t));
  if (!b_one.p) return set_error(c, GM_E_NOMEM, "PIC scratch");
  {
    const int64_t zero = 0;
    const int32_t dimR = R;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(b_one.p, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
    GM_CUDA_CHECK(c, cudaMemcpyAsync((char*)b_one.p + sizeof(int64_t), &dimR, sizeof(dimR),
                                     cudaMemcpyHostToDevice, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));  // the host values above are stack locals
  }
  const int64_t* one_off = (const int64_t*)b_one.p;
  const int32_t* one_dim = (const int32_t*)((char*)b_one.p + sizeof(int64_t));
  GM_PROF(c, "k_pic_chol");
  k_pic_chol<<<1, 256, 0, st>>>(Lu, one_off, one_dim, c->d_flags);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_arow");
  k_pic_arow<<<grid_for(c, n), 128, 0, st>>>(n, R, Lu, Kku, A);
  GM_LAUNCH_CHECK(c);
  // ---- blocks: C_k, its factor, X_k and yv_k
  if (coff[nb] > 0) {
    GM_PROF(c, "k_pic_cmat");
    k_pic_cmat<<<grid_for(c, coff[nb]), 128, 0, st>>>(nb, d_coff, d_boff, R, d_bidx, c->row_ptr,
                                                      c->col, (const double*)c->val, A, Kku,
                                                      c->obs_sigma, C);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_pic_chol");
    k_pic_chol<<<nb, 256, 0, st>>>(C, d_coff, d_dims, c->d_flags);
    GM_LAUNCH_CHECK(c);
  }
  GM_PROF(c, "k_pic_y");
  k_pic_y<<<grid_for(c, n), 128, 0, st>>>(n, R, d_bidx, c->obs, c->prior_m, A, mu_u, yv);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(X, A, n * (int64_t)R * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
  GM_PROF(c, "k_pic_fsolve");
  k_pic_fsolve<<<grid_for(c, (int64_t)nb * (R + 1)), 128, 0, st>>>(nb, R, d_coff, d_boff, C, X,
                                                                    yv);
  GM_LAUNCH_CHECK(c);
  // ---- posterior of u
  GM_PROF(c, "k_pic_lambda");
  k_pic_lambda<<<grid_for(c, RR + R), 128, 0, st>>>(n, R, X, yv, Lam, eta);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_inverse");
  k_pic_inverse<<<grid_for(c, R), 128, 0, st>>>(R, Lu, Kinv);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_prec");
  k_pic_prec<<<grid_for(c, RR + R), 128, 0, st>>>(R, Kinv, Lam, mu_u, eta, P, h);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_chol");
  k_pic_chol<<<1, 256, 0, st>>>(P, one_off, one_dim, c->d_flags);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_mean");
  k_pic_mean<<<1, 32, 0, st>>>(R, P, h, mean);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_inverse");
  k_pic_inverse<<<grid_for(c, R), 128, 0, st>>>(R, P, cov);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  dev_free_now(c, qcol.p, qcol.bytes);
  return GM_OK;
}

}  // namespace gm
