// Mean function of the dust density and its hyperparameters (Sect. 2
// learning phase; Sect. 5 set-up).
//
// Sect. 5 takes the mean extinction pseudo-density to be an exponential disc
// (scale length L, scale height H, pseudo-density rho0 at the Sun) plus a
// Gaussian bump along the line of sight standing in for a spiral arm (distance
// s_b, total extinction A_b, width w fixed), five hyperparameters with
// log-normal hyperpriors.  With the Sun at R_sun from the Galactic centre and
// heliocentric x towards it, the mean density is
//   rho(x) = rho0 exp(-(R(x) - R_sun)/L - |z|/H) + A_b N(|x|; s_b, w^2),
// R(x) = |(R_sun - x_1, x_2)|, and the mean extinction of a star is its line
// integral; the prior mean of a = ln A is the lognormal moment match
//   m_i = ln E[A_i] - K_ii / 2,
// with K the covariance of the stationary relative fluctuations (so the
// hyperparameters enter the prior mean only).  The disc integral uses a
// 64-node Gauss-Legendre rule along the sightline (the integrand is smooth),
// the bump its closed form with the normal distribution function; the
// derivatives with respect to ln theta come with it.
//
// Learning.  With the likelihood Gaussian in a (the simplified case of
// Sect. 4.1) the marginal likelihood is exact, atilde ~ N(m(theta), K +
// Sigma), and the log posterior of phi = ln theta is, up to a constant,
//   -1/2 r^T (K + Sigma)^-1 r + ln N(phi; mu, s^2),   r = atilde - m,
// with gradient g = J^T (K + Sigma)^-1 r - (phi - mu)/s^2, J = dm/dphi.
// (K + Sigma)^-1 r is the alpha of the posterior-mean solve at the exact
// sites tau = 1/sigma^2, nu = atilde/sigma^2 with prior mean m.  The mode is
// found by Newton steps: Hessian by central differences of g (step 1e-4 in
// phi), symmetrised, shifted by d I (d doubling from min 1/s^2) until its
// Cholesky factor exists; a step that does not raise the log posterior is
// halved.  The Laplace covariance of phi is the inverse Hessian at the mode.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kMfNodes = 64;

struct MeanFn {
  double L, H, rho0, sb, Ab, rsun, w;
};

static MeanFn mean_fn_of(const double* theta, double rsun, double w) {
  return MeanFn{theta[0], theta[1], theta[2], theta[3], theta[4], rsun, w};
}

// E[A] along (u, s) and its derivatives with respect to ln theta_k:
// out = {E, dE/dlnL, dE/dlnH, dE/dlnrho0, dE/dlns_b, dE/dlnA_b}
__device__ __forceinline__ void mean_fn_eval(const MeanFn& f, double s, double ux, double uy,
                                             double uz, const double* __restrict__ zeta,
                                             const double* __restrict__ wq, double out[6]) {
  double e = 0, eL = 0, eH = 0;
  for (int q = 0; q < kMfNodes; ++q) {
    const double t = s * zeta[q];
    const double dR = hypot(f.rsun - t * ux, t * uy) - f.rsun;
    const double az = fabs(t * uz);
    const double d = wq[q] * f.rho0 * exp(-dR / f.L - az / f.H);
    e += d;
    eL += d * (dR / f.L);
    eH += d * (az / f.H);
  }
  e *= s;
  eL *= s;
  eH *= s;
  const double a = (s - f.sb) / f.w, a0 = -f.sb / f.w;
  const double inv_sqrt_2pi = 0.3989422804014327;
  const double Eb = f.Ab * (normcdf(a) - normcdf(a0));
  out[0] = e + Eb;
  out[1] = eL;
  out[2] = eH;
  out[3] = e;
  out[4] = f.sb * f.Ab * inv_sqrt_2pi * (exp(-0.5 * a0 * a0) - exp(-0.5 * a * a)) / f.w;
  out[5] = Eb;
}

// m = ln E[A] - kss/2 per point; J (column k at J + k n, may be null) = d m / d ln theta_k
__global__ void k_mean_fn(int64_t n, MeanFn f, const double* __restrict__ s,
                          const double* __restrict__ ux, const double* __restrict__ uy,
                          const double* __restrict__ uz, const double* __restrict__ kss,
                          const double* __restrict__ zeta, const double* __restrict__ wq,
                          double* __restrict__ m, double* __restrict__ J,
                          unsigned* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double o[6];
    mean_fn_eval(f, s[i], ux[i], uy[i], uz[i], zeta, wq, o);
    const double E = o[0];
    if (!(E > 0) || !isfinite(E)) atomicOr(flags, kFlagNonFinite);
    m[i] = log(E) - 0.5 * kss[i];
    if (J)
      for (int k = 0; k < 5; ++k) J[k * n + i] = o[k + 1] / E;
  }
}

// exact sites of a likelihood Gaussian in a: tau = 1/sigma^2, nu = atilde/sigma^2
__global__ void k_exact_sites(int64_t n, const double* __restrict__ obs,
                              const double* __restrict__ sig, double* __restrict__ tau,
                              double* __restrict__ nu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double p = 1.0 / (sig[i] * sig[i]);
    tau[i] = p;
    nu[i] = obs[i] * p;
  }
}

// the constant-density prior mean: ln(rho_bar s) - K_ii/2 (lognormal form)
// or - sigma2/2 (first-order form)
__global__ void k_const_mean(int64_t n, double log_rho_bar, int form, double sigma2,
                             const double* __restrict__ s, const double* __restrict__ kdiag,
                             double* __restrict__ m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m[i] = log_rho_bar + log(s[i]) - (form == GM_FORM_LOGNORMAL ? 0.5 * kdiag[i] : 0.5 * sigma2);
}

constexpr int kLdThreads = 256;

// per-block partial sums (fixed order) of r . alpha and J_k . alpha, r = obs - m
__global__ void __launch_bounds__(kLdThreads) k_learn_dots(int64_t n, const double* __restrict__ obs,
                                                          const double* __restrict__ m,
                                                          const double* __restrict__ alpha,
                                                          const double* __restrict__ J,
                                                          double* __restrict__ part) {
  __shared__ double sh[6][kLdThreads / 32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = alpha[i];
    acc[0] += (obs[i] - m[i]) * a;
    for (int k = 0; k < 5; ++k) acc[k + 1] += J[k * n + i] * a;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) sh[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0;
    for (int q = 0; q < kLdThreads / 32; ++q) t += sh[threadIdx.x][q];
    part[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

static gm_status ensure_rule(gm_ctx* c) {
  if (c->mf_gl.p) return GM_OK;
  if (!ensure(c, c->mf_gl, 2 * kMfNodes * sizeof(double)))
    return set_error(c, GM_E_NOMEM, "mean-function rule");
  double x[kMfNodes], w[kMfNodes], h[2 * kMfNodes];
  gauss_legendre(kMfNodes, x, w);
  for (int q = 0; q < kMfNodes; ++q) {
    h[q] = 0.5 * (1.0 + x[q]);
    h[kMfNodes + q] = 0.5 * w[q];
  }
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->mf_gl.p, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

gm_status mean_fn_apply(gm_ctx* c, int64_t n, const double* s, const double* ux,
                        const double* uy, const double* uz, const double* kss, double* m,
                        double* J) {
  if (n == 0) return GM_OK;
  gm_status st = ensure_rule(c);
  if (st != GM_OK) return st;
  const double* z = (const double*)c->mf_gl.p;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 128), 8 * sm_count(c)));
  GM_PROF(c, "k_mean_fn");
  k_mean_fn<<<g, 128, 0, c->stream>>>(n, mean_fn_of(c->mean_theta, c->mean_rsun, c->mean_w), s,
                                      ux, uy, uz, kss, z, z + kMfNodes, m, J, c->d_flags);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

namespace {

struct Eval {
  double g[5];
  double lp;
};

// 5 x 5 Cholesky in place (lower); false if not positive definite
bool chol5(double A[25]) {
  for (int j = 0; j < 5; ++j) {
    double d = A[j * 5 + j];
    for (int k = 0; k < j; ++k) d -= A[j * 5 + k] * A[j * 5 + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[j * 5 + j] = d;
    for (int i = j + 1; i < 5; ++i) {
      double v = A[i * 5 + j];
      for (int k = 0; k < j; ++k) v -= A[i * 5 + k] * A[j * 5 + k];
      A[i * 5 + j] = v / d;
    }
  }
  return true;
}

// x = A^-1 b with the Cholesky factor of A (lower)
void chol5_solve(const double Lf[25], const double* b, double* x) {
  double y[5];
  for (int i = 0; i < 5; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= Lf[i * 5 + k] * y[k];
    y[i] = v / Lf[i * 5 + i];
  }
  for (int i = 4; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < 5; ++k) v -= Lf[k * 5 + i] * x[k];
    x[i] = v / Lf[i * 5 + i];
  }
}

}  // namespace

// Log posterior (theta-dependent part) and its gradient at phi; leaves the
// context's prior mean at m(exp phi) and alpha, mu for it.
static gm_status learn_eval(gm_ctx* c, const double phi[5], const double mu[5],
                            const double s2[5], Eval* out) {
  for (int k = 0; k < 5; ++k) c->mean_theta[k] = std::exp(phi[k]);
  double* J = (double*)c->mf_J.p;
  gm_status st = mean_fn_apply(c, c->n, c->s, c->ux, c->uy, c->uz, c->kdiag, c->prior_m, J);
  if (st != GM_OK) return st;
  st = posterior_mean_only(c);
  if (st != GM_OK) return st;
  const int G = 2 * sm_count(c);
  double* part = (double*)c->mf_part.p;
  GM_PROF(c, "k_learn_dots");
  k_learn_dots<<<G, kLdThreads, 0, c->stream>>>(c->n, c->obs, c->prior_m, c->alpha, J, part);
  GM_LAUNCH_CHECK(c);
  std::vector<double> hp(6 * (size_t)G);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  st = read_flags(c);
  if (st != GM_OK) return st;
  double d[6];
  for (int k = 0; k < 6; ++k) {
    d[k] = 0;
    for (int b = 0; b < G; ++b) d[k] += hp[k * (size_t)G + b];
  }
  double lp = -0.5 * d[0];
  for (int k = 0; k < 5; ++k) {
    out->g[k] = d[k + 1] - (phi[k] - mu[k]) / s2[k];
    lp += -0.5 * (phi[k] - mu[k]) * (phi[k] - mu[k]) / s2[k] - 0.5 * std::log(2 * M_PI * s2[k]);
  }
  if (!std::isfinite(lp)) return set_error(c, GM_E_NONFINITE, "log posterior is not finite");
  out->lp = lp;
  return GM_OK;
}

// Negative Hessian of the log posterior at phi (central differences of the
// gradient), symmetrised and shifted until positive definite; its Cholesky
// factor in Lf.
static gm_status learn_hessian(gm_ctx* c, const double phi[5], const double mu[5],
                               const double s2[5], double Hm[25], double Lf[25]) {
  const double h = 1e-4;
  for (int k = 0; k < 5; ++k) {
    double p[5], q[5];
    for (int j = 0; j < 5; ++j) p[j] = q[j] = phi[j];
    p[k] += h;
    q[k] -= h;
    Eval a, b;
    gm_status st = learn_eval(c, p, mu, s2, &a);
    if (st == GM_OK) st = learn_eval(c, q, mu, s2, &b);
    if (st != GM_OK) return st;
    for (int j = 0; j < 5; ++j) Hm[j * 5 + k] = -(a.g[j] - b.g[j]) / (2 * h);
  }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < i; ++j) Hm[i * 5 + j] = Hm[j * 5 + i] = 0.5 * (Hm[i * 5 + j] + Hm[j * 5 + i]);
  double dmin = 1.0 / s2[0];
  for (int k = 1; k < 5; ++k) dmin = std::min(dmin, 1.0 / s2[k]);
  double shift = 0;
  for (int tries = 0; tries < 80; ++tries) {
    for (int i = 0; i < 25; ++i) Lf[i] = Hm[i];
    for (int i = 0; i < 5; ++i) Lf[i * 5 + i] += shift;
    if (chol5(Lf)) {
      for (int i = 0; i < 5; ++i) Hm[i * 5 + i] += shift;
      return GM_OK;
    }
    shift = shift > 0 ? 2 * shift : dmin;
  }
  return set_error(c, GM_E_NONFINITE, "Hessian of the log posterior");
}

}  // namespace gm

using namespace gm;

extern "C" gm_status gm_set_mean_fn(gm_ctx* c, const double* theta, double r_sun_pc,
                                    double bump_width_pc) {
  if (!c) return GM_E_INVAL;
  if (!theta) {  // back to the constant mean density rho_bar
    c->mean_fn_on = false;
    if (c->built) {
      GM_PROF(c, "k_const_mean");
      k_const_mean<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c->n, 256),
                                                                  8 * sm_count(c))),
                     256, 0, c->stream>>>(c->n, std::log(c->cfg.rho_bar), c->cfg.form,
                                          c->cfg.sigma2, c->s, c->kdiag, c->prior_m);
      GM_LAUNCH_CHECK(c);
      gm_status st = read_flags(c);
      if (st != GM_OK) return st;
      c->post_valid = false;
    }
    return GM_OK;
  }
  for (int k = 0; k < 5; ++k)
    if (!(theta[k] > 0) || !std::isfinite(theta[k])) return GM_E_INVAL;
  if (!(r_sun_pc > 0) || !(bump_width_pc > 0)) return GM_E_INVAL;
  if (c->n_fields > 1) return set_error(c, GM_E_STATE, "mean function needs one field");
  c->launches = 0;
  for (int k = 0; k < 5; ++k) c->mean_theta[k] = theta[k];
  c->mean_rsun = r_sun_pc;
  c->mean_w = bump_width_pc;
  c->mean_fn_on = true;
  if (c->built) {
    gm_status st = mean_fn_apply(c, c->n, c->s, c->ux, c->uy, c->uz, c->kdiag, c->prior_m, nullptr);
    if (st == GM_OK) st = read_flags(c);
    if (st != GM_OK) return st;
    c->post_valid = false;
  }
  return GM_OK;
}

extern "C" gm_status gm_learn_mean(gm_ctx* c, const double* theta0, const double* prior_mean,
                                   const double* prior_sd, double r_sun_pc, double bump_width_pc,
                                   int32_t max_iter, double tol, double* theta_out,
                                   double* cov_out, double* log_post_out, int32_t* iters_out) {
  if (!c || !theta0 || !prior_mean || !prior_sd || !theta_out || max_iter < 1 || !(tol > 0))
    return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must precede gm_learn_mean");
  if (c->cfg.likelihood != GM_LIK_GAUSS_IN_LNA)
    return set_error(c, GM_E_INVAL, "mean learning needs the likelihood Gaussian in ln A");
  if (c->cfg.form != GM_FORM_LOGNORMAL)
    return set_error(c, GM_E_INVAL, "mean learning needs the lognormal form");
  double mu[5], s2[5], phi[5];
  for (int k = 0; k < 5; ++k) {
    if (!(prior_mean[k] > 0) || !(prior_sd[k] > 0) || !(theta0[k] > 0)) return GM_E_INVAL;
    s2[k] = std::log1p((prior_sd[k] / prior_mean[k]) * (prior_sd[k] / prior_mean[k]));
    mu[k] = std::log(prior_mean[k]) - 0.5 * s2[k];
    phi[k] = std::log(theta0[k]);
  }
  gm_status st = gm_set_mean_fn(c, theta0, r_sun_pc, bump_width_pc);
  if (st != GM_OK) return st;
  c->launches = 0;
  // The Hessian comes from differences of gradients 1e-4 apart in phi, so the
  // gradients' solves run to 1e-12 (FP32 contexts: by the FP64-residual
  // refinement of the mean solve); the context's tolerance is restored after.
  struct TolGuard {
    gm_ctx* c;
    double tol;
    ~TolGuard() { c->cfg.cg_tol = tol; }
  } guard{c, c->cfg.cg_tol};
  c->cfg.cg_tol = std::min(c->cfg.cg_tol, 1e-12);
  const int G = 2 * sm_count(c);
  if (!ensure(c, c->mf_J, (size_t)5 * c->n * sizeof(double)) ||
      !ensure(c, c->mf_part, (size_t)6 * G * sizeof(double)))
    return set_error(c, GM_E_NOMEM, "mean learning scratch");
  GM_PROF(c, "k_exact_sites");
  k_exact_sites<<<(int)std::min<int64_t>(ceil_div(c->n, 256), 8 * sm_count(c)), 256, 0,
                  c->stream>>>(c->n, c->obs, c->obs_sigma, c->tau, c->nu);
  GM_LAUNCH_CHECK(c);
  Eval e;
  st = learn_eval(c, phi, mu, s2, &e);
  if (st != GM_OK) return st;
  double Hm[25], Lf[25];
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    st = learn_hessian(c, phi, mu, s2, Hm, Lf);
    if (st != GM_OK) return st;
    double step[5];
    chol5_solve(Lf, e.g, step);
    double lam = 1.0, ph[5];
    Eval en;
    for (;;) {
      for (int k = 0; k < 5; ++k) ph[k] = phi[k] + lam * step[k];
      st = learn_eval(c, ph, mu, s2, &en);
      if (st != GM_OK) return st;
      if (en.lp >= e.lp || lam < 1e-6) break;
      lam *= 0.5;
    }
    double mx = 0;
    for (int k = 0; k < 5; ++k) {
      mx = std::max(mx, std::fabs(lam * step[k]));
      phi[k] = ph[k];
    }
    e = en;
    if (mx < tol) break;
  }
  it = std::min(it, (int)max_iter);
  st = learn_hessian(c, phi, mu, s2, Hm, Lf);
  if (st != GM_OK) return st;
  // leave the context at the mode: prior mean m(theta), alpha and mu for it
  st = learn_eval(c, phi, mu, s2, &e);
  if (st != GM_OK) return st;
  for (int k = 0; k < 5; ++k) theta_out[k] = std::exp(phi[k]);
  if (cov_out) {
    for (int k = 0; k < 5; ++k) {
      double ek[5] = {0, 0, 0, 0, 0}, col[5];
      ek[k] = 1.0;
      chol5_solve(Lf, ek, col);
      for (int j = 0; j < 5; ++j) cov_out[j * 5 + k] = col[j];
    }
  }
  if (log_post_out) *log_post_out = e.lp;
  if (iters_out) *iters_out = it;
  prof_collect(c);
  c->post_valid = false;  // the variances are not recomputed
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}
