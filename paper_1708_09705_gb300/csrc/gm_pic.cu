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

// Factors of the last PIC posterior, kept for prediction.
struct PicState {
  int R = 0, nb = 0;
  int64_t n = 0;
  Buffer i64;  // boff (nb + 1), coff (nb + 1), bidx (n)
  Buffer i32;  // dims (nb)
  Buffer d;    // Lu (R^2), mean (R), cov (R^2), mu_u (R), us, ux, uy, uz (R),
               // A, Kku (n R), C factors (sum N_k^2)
  std::vector<int64_t> h_boff, h_coff;
  int64_t *boff = nullptr, *coff = nullptr, *bidx = nullptr;
  int32_t* dims = nullptr;
  double *Lu = nullptr, *mean = nullptr, *cov = nullptr, *mu_u = nullptr, *us = nullptr,
         *ux = nullptr, *uy = nullptr, *uz = nullptr, *A = nullptr, *Kku = nullptr, *C = nullptr;
  int max_block = 0;
  bool ready = false;  // set once the posterior is complete
};

void pic_free(gm_ctx* c) {
  if (!c->pic) return;
  PicState* P = c->pic;
  for (Buffer* b : {&P->i64, &P->i32, &P->d})
    if (b->p) dev_free_now(c, b->p, b->bytes);
  delete P;
  c->pic = nullptr;
}

bool pic_ready(gm_ctx* c) { return c->pic && c->pic->ready; }
const double* pic_mean(gm_ctx* c) { return c->pic ? c->pic->mean : nullptr; }
const double* pic_cov(gm_ctx* c) { return c->pic ? c->pic->cov : nullptr; }
int pic_blocks(gm_ctx* c) { return c->pic ? c->pic->nb : 0; }
int pic_inducing(gm_ctx* c) { return c->pic ? c->pic->R : 0; }

gm_status pic_posterior(gm_ctx* c, int R, const double* us, const double* ux, const double* uy,
                        const double* uz, const int32_t* h_block_int, int nb) {
  const int64_t n = c->n;
  pic_free(c);
  PicState* S = new (std::nothrow) PicState();
  if (!S) return set_error(c, GM_E_NOMEM, "PIC state");
  c->pic = S;
  S->R = R;
  S->nb = nb;
  S->n = n;
  // ---- block lists (host): stars of block k in internal order
  S->h_boff.resize(nb + 1);
  S->h_coff.resize(nb + 1);
  std::vector<int64_t> bidx(n);
  std::vector<int32_t> rowpos(n), dims(nb);
  if (!gmpic::block_lists(n, h_block_int, nb, kMaxPicBlock, S->h_boff.data(), S->h_coff.data(),
                          bidx.data(), rowpos.data(), dims.data())) {
    pic_free(c);
    return set_error(c, GM_E_INVAL, "a sub-catalogue has more than 8192 stars");
  }
  for (int k = 0; k < nb; ++k) S->max_block = std::max(S->max_block, (int)dims[k]);
  const int64_t RR = (int64_t)R * R;
  const int64_t npair = (int64_t)R * (R + 1) / 2;
  const int64_t ncf = S->h_coff[nb];
  if (!ensure(c, S->i64, (size_t)(2 * (nb + 1) + n) * sizeof(int64_t)) ||
      !ensure(c, S->i32, (size_t)std::max(nb, 1) * sizeof(int32_t)) ||
      !ensure(c, S->d, (size_t)(2 * RR + 7 * R + 2 * n * (int64_t)R + ncf) * sizeof(double))) {
    pic_free(c);
    return set_error(c, GM_E_NOMEM, "PIC state");
  }
  S->boff = (int64_t*)S->i64.p;
  S->coff = S->boff + nb + 1;
  S->bidx = S->coff + nb + 1;
  S->dims = (int32_t*)S->i32.p;
  S->Lu = (double*)S->d.p;
  S->mean = S->Lu + RR;
  S->cov = S->mean + R;
  S->mu_u = S->cov + RR;
  S->us = S->mu_u + R;
  S->ux = S->us + R;
  S->uy = S->ux + R;
  S->uz = S->uy + R;
  S->A = S->uz + R;
  S->Kku = S->A + n * (int64_t)R;
  S->C = S->Kku + n * (int64_t)R;
  // scratch of this call: Kuu, Kinv, Lam, P (R x R); eta, h (R); pair inputs
  // (4 npair); X (n x R); yv (n); rowpos (n)
  ScopedDev b_d(c, (size_t)(4 * RR + 2 * R + 4 * npair + n * (int64_t)R + n) * sizeof(double));
  ScopedDev b_r(c, (size_t)n * sizeof(int32_t));
  ScopedDev b_q(c, (size_t)(R + 1) * sizeof(int64_t));
  ScopedDev b_one(c, sizeof(int64_t) + sizeof(int32_t));
  if (!b_d.p || !b_r.p || !b_q.p || !b_one.p) return set_error(c, GM_E_NOMEM, "PIC arrays");
  double* Kuu = (double*)b_d.p;
  double *Kinv = Kuu + RR, *Lam = Kinv + RR, *P = Lam + RR, *eta = P + RR, *h = eta + R;
  double *psi = h + R, *psj = psi + npair, *pch = psj + npair, *pk = pch + npair;
  double *X = pk + npair, *yv = X + n * (int64_t)R;
  int32_t* d_rowpos = (int32_t*)b_r.p;
  double *Lu = S->Lu, *A = S->A, *Kku = S->Kku, *C = S->C, *mu_u = S->mu_u;
  cudaStream_t st = c->stream;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S->boff, S->h_boff.data(), (nb + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S->coff, S->h_coff.data(), (nb + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S->bidx, bidx.data(), n * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(d_rowpos, rowpos.data(), n * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S->dims, dims.data(), nb * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  for (const double* src : {us, ux, uy, uz}) {
    double* dst = src == us ? S->us : src == ux ? S->ux : src == uy ? S->uy : S->uz;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(dst, src, R * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  GM_CUDA_CHECK(c, cudaMemsetAsync(Kku, 0, n * (int64_t)R * sizeof(double), st));
  // ---- K_ku: the inducing points' neighbour CSR over the stars
  int64_t* qptr = (int64_t*)b_q.p;
  Buffer qcol;
  int64_t qnnz = 0;
  gm_status s = neighbour_csr(c, R, us, ux, uy, uz, nullptr, false, qptr, qcol, &qnnz, nullptr);
  if (s != GM_OK) return s;
  ScopedDev b_qc(c, qcol.p, qcol.bytes, ScopedDev::Adopt{});  // released on every return
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
  if (ncf > 0) {
    GM_PROF(c, "k_pic_cmat");
    k_pic_cmat<<<grid_for(c, ncf), 128, 0, st>>>(nb, S->coff, S->boff, R, S->bidx, c->row_ptr,
                                                 c->col, (const double*)c->val, A, Kku,
                                                 c->obs_sigma, C);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_pic_chol");
    k_pic_chol<<<nb, 256, 0, st>>>(C, S->coff, S->dims, c->d_flags);
    GM_LAUNCH_CHECK(c);
  }
  GM_PROF(c, "k_pic_y");
  k_pic_y<<<grid_for(c, n), 128, 0, st>>>(n, R, S->bidx, c->obs, c->prior_m, A, mu_u, yv);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(X, A, n * (int64_t)R * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
  GM_PROF(c, "k_pic_fsolve");
  k_pic_fsolve<<<grid_for(c, (int64_t)nb * (R + 1)), 128, 0, st>>>(nb, R, S->coff, S->boff, C,
                                                                    X, yv);
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
  k_pic_mean<<<1, 32, 0, st>>>(R, P, h, S->mean);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pic_inverse");
  k_pic_inverse<<<grid_for(c, R), 128, 0, st>>>(R, P, S->cov);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  S->ready = true;
  return GM_OK;
}

// ---------------------------------------------------------------- prediction
__global__ void k_pic_qpairs(int64_t np, int R, const double* __restrict__ qs,
                             const double* __restrict__ qx, const double* __restrict__ qy,
                             const double* __restrict__ qz, const double* __restrict__ us,
                             const double* __restrict__ ux, const double* __restrict__ uy,
                             const double* __restrict__ uz, double* __restrict__ si,
                             double* __restrict__ sj, double* __restrict__ ch) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x)
    gmpic::qpair(p, R, qs, qx, qy, qz, us, ux, uy, uz, si, sj, ch);
}

__global__ void k_pic_ksu(int64_t np, double inv_cut, int taper, const double* __restrict__ si,
                          const double* __restrict__ sj, const double* __restrict__ ch,
                          double* __restrict__ kp) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x)
    kp[p] = gmpic::ksu_entry(p, inv_cut, taper, si, sj, ch, kp);
}

// One thread per query of the chunk [q0, q0 + nc).
__global__ void k_pic_point(int64_t q0, int64_t nc, int R, int maxN,
                            const int32_t* __restrict__ qblk, const int64_t* __restrict__ boff,
                            const int64_t* __restrict__ coff, const int64_t* __restrict__ bidx,
                            const double* __restrict__ Lu, const double* __restrict__ Cf,
                            const double* __restrict__ A, const double* __restrict__ Kku,
                            const double* __restrict__ mu_u, const double* __restrict__ pmean,
                            const double* __restrict__ pcov, const double* __restrict__ obs,
                            const double* __restrict__ prior_m, const double* __restrict__ ksu,
                            const double* __restrict__ kss, const double* __restrict__ ms,
                            const int64_t* __restrict__ qptr, const int32_t* __restrict__ qcol,
                            const double* __restrict__ qval, double* __restrict__ scratch,
                            double* __restrict__ mean, double* __restrict__ var) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc) return;
  const int64_t q = q0 + t;
  double* w = scratch + t * (3 * (int64_t)R + 2 * (int64_t)maxN);
  gmpic::pic_point(R, qblk[q], boff, coff, bidx, Lu, Cf, A, Kku, mu_u, pmean, pcov, obs, prior_m,
                   ksu + t * R, kss[q], ms[q], qptr[q], qptr[q + 1], qcol, qval, w, w + R,
                   w + 2 * R, w + 3 * R, w + 3 * R + maxN, mean + q, var + q);
}

gm_status pic_predict(gm_ctx* c, int64_t nq, const double* qs, const double* qx,
                      const double* qy, const double* qz, const int32_t* qblk, const double* kss,
                      const double* ms, const int64_t* qptr, const int32_t* qcol,
                      const double* qval, double* mean, double* var) {
  PicState* S = c->pic;
  const int R = S->R;
  const int maxN = std::max(S->max_block, 1);
  // queries per chunk: K_su pairs (4 R doubles each) and the scratch
  // (3 R + 2 maxN doubles each) within about 1 GB
  const int64_t per = 4 * (int64_t)R + 3 * (int64_t)R + 2 * (int64_t)maxN;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)(1 << 27) / per));
  ScopedDev buf(c, (size_t)chunk * per * sizeof(double));
  if (!buf.p) return set_error(c, GM_E_NOMEM, "PIC prediction scratch");
  double* si = (double*)buf.p;
  double *sj = si + chunk * R, *ch = sj + chunk * R, *kp = ch + chunk * R, *w = kp + chunk * R;
  cudaStream_t st = c->stream;
  for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
    const int64_t nc = std::min(chunk, nq - q0);
    const int64_t np = nc * R;
    GM_PROF(c, "k_pic_qpairs");
    k_pic_qpairs<<<grid_for(c, np), 128, 0, st>>>(np, R, qs + q0, qx + q0, qy + q0, qz + q0,
                                                  S->us, S->ux, S->uy, S->uz, si, sj, ch);
    GM_LAUNCH_CHECK(c);
    gm_status s = pairlist_quadrature(c, np, si, sj, ch, kp);
    if (s != GM_OK) return s;
    GM_PROF(c, "k_pic_ksu");
    k_pic_ksu<<<grid_for(c, np), 128, 0, st>>>(np, 1.0 / c->cfg.cutoff_pc, c->cfg.taper, si, sj,
                                               ch, kp);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_pic_point");
    k_pic_point<<<(unsigned)ceil_div(nc, 128), 128, 0, st>>>(
        q0, nc, R, maxN, qblk, S->boff, S->coff, S->bidx, S->Lu, S->C, S->A, S->Kku, S->mu_u,
        S->mean, S->cov, c->obs, c->prior_m, kp, kss, ms, qptr, qcol, qval, w, mean, var);
    GM_LAUNCH_CHECK(c);
  }
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  return GM_OK;
}

}  // namespace gm
