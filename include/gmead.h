/*
 * gmead.h -- C ABI of libgmead, the GPU hot path of Gaussian-process 3-D
 * extinction mapping with expectation propagation (Sale & Magorrian 2018,
 * "Large-scale three-dimensional Gaussian process extinction mapping").
 *
 * The library computes, on one CUDA GPU (sm_103a):
 *   - the sparse covariance K of the stars' log-extinctions a_i = ln A_i:
 *     the covariance of the log-density integrated along both sightlines
 *     (Sect. 3), for a log-density whose fluctuations follow a Kolmogorov
 *     spectrum truncated at the outer scale (Sect. 1), evaluated by
 *     Gauss-Legendre quadrature on each sightline, with pairs whose 3-D
 *     separation exceeds a cutoff dropped (compactly supported taper);
 *   - parallel expectation propagation with one Gaussian site per star
 *     (App. A.2: cavity, tilted distribution, moment matching), whose
 *     posterior marginals come from preconditioned conjugate-gradient
 *     solves driven by sparse matrix products;
 *   - the posterior predictive of a at query points (Sect. 2 eq. cond_GP0,
 *     Sect. 3.1 eq. map_dist), jointly for pairs or sightlines of points;
 *   - the Sect. 5 products built on it: the extinction pseudo-density, and
 *     samples of each sightline's predictive conditioned on dA/ds >= 0.
 *
 * Conventions for every call:
 *   - Angles in radians, distances in pc, extinctions in mag.  Returned
 *     moments are those of the natural log of the extinction.
 *   - Array arguments may be host or device pointers; the library detects
 *     which with cudaPointerGetAttributes.  Inputs are copied: the caller
 *     keeps ownership and may free them when the call returns.  Outputs go to
 *     caller-allocated arrays of the stated length.
 *   - Arrays are indexed in the caller's star order.  Internally the stars
 *     are renumbered by a spatial sort; gm_get_perm exposes that order.
 *   - Every call returns a gm_status; no C++ exception crosses the ABI.  A
 *     human-readable detail of the last failure is kept per context
 *     (gm_last_error).  Kernels never trap: they raise status flags that the
 *     host reads.
 *   - All work is issued on the context's stream.  Calls that return host
 *     data synchronise that stream.  A context must not be used from two
 *     threads at once.
 */
#ifndef GMEAD_H
#define GMEAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_ctx gm_ctx;

typedef enum {
  GM_OK = 0,
  GM_E_INVAL = 1,      /* bad argument (null pointer, size, config value)   */
  GM_E_NOMEM = 2,      /* device allocation failed                          */
  GM_E_CUDA = 3,       /* CUDA runtime error (detail in gm_last_error)      */
  GM_E_NOT_SPD = 4,    /* CG met p^T B p <= 0, or a sightline covariance
                          has no Cholesky factor: not positive definite     */
  GM_E_NOCONV = 5,     /* CG hit its iteration cap above tolerance, or a
                          sampler step its wall-hit limit                   */
  GM_E_NONFINITE = 6,  /* a NaN or Inf appeared in K, the solves or sites   */
  GM_E_TIMEOUT = 7,    /* a bounded device wait gave up                     */
  GM_E_STATE = 8       /* call out of order (e.g. sweep before build_cov)   */
} gm_status;

/* Arithmetic of the covariance values, quadrature and CG inner iterations.
 * Site updates and the moments they use are always FP64. */
enum { GM_PREC_FP64 = 0, GM_PREC_FP32 = 1 };
/* Log-extinction moments from the density moments: lognormal moment match
 * (K = log1p(I/(s_i s_j)), m = ln(rho_bar s) - K_ii/2) or first order. */
enum { GM_FORM_LOGNORMAL = 0, GM_FORM_LINEAR = 1 };
/* Sparsification: Wendland psi_{3,1} taper (keeps K positive definite) or a
 * hard cutoff (literal dropping; may be indefinite -> GM_E_NOT_SPD). */
enum { GM_TAPER_WENDLAND = 0, GM_TAPER_HARD = 1 };
/* Source of the covariance entries: the sightline quadrature, or the learned
 * surrogate (gm_surrogate_*) with quadrature fallback beyond the gate. */
enum { GM_COV_QUADRATURE = 0, GM_COV_SURROGATE = 1 };
/* Per-star likelihood: A_obs ~ N(exp(a), sigma^2) or a_obs ~ N(a, sigma^2). */
enum { GM_LIK_GAUSS_IN_A = 0, GM_LIK_GAUSS_IN_LNA = 1 };
/* Node rule of the sightline double integral (Sect. 3): n_nodes-point
 * Gauss-Legendre on each sightline, or the band rule (composite
 * Gauss-Legendre in d = t - t' and m = (t + t')/2, panels graded towards the
 * cusp of the kernel at zero separation, truncated at 40 outer scales),
 * which converges where the distance is many outer scales (the global rule's
 * nodes are s / n_nodes apart). */
enum { GM_QUAD_GL = 0, GM_QUAD_BAND = 1 };

typedef struct {
  double sigma2;          /* variance of the log-density GP (> 0)             */
  double outer_scale_pc;  /* outer (injection) scale L0; k0 = 1/L0 (> 0)      */
  double rho_bar;         /* mean extinction per pc, E[exp f] (> 0)           */
  double cutoff_pc;       /* pairs farther apart in 3-D are dropped (> 0)     */
  int32_t n_nodes;        /* Gauss-Legendre nodes per sightline, 2..128       */
  int32_t form;           /* GM_FORM_*                                        */
  int32_t taper;          /* GM_TAPER_*                                       */
  int32_t precision;      /* GM_PREC_*                                        */
  int32_t likelihood;     /* GM_LIK_*                                         */
  int32_t cg_max_iter;    /* cap on CG iterations per solve (> 0)             */
  double damping;         /* EP damping eta in (0, 1]                         */
  double vc_floor;        /* floor on the cavity variance (>= 0)              */
  double cg_tol;          /* CG stops at ||r|| <= cg_tol ||b|| (> 0); FP32
                             variance panels use max(cg_tol, 1e-5)            */
  int32_t rhs_panel;      /* right-hand sides per variance panel, 0 = auto    */
  int32_t warm_start;     /* 1: start each sweep's variance CG from the
                             previous sweep's solutions (same results within
                             cg_tol; resume from saved sites is then equal
                             within cg_tol, not bit for bit); 0: cold start   */
  int32_t cov_source;     /* GM_COV_QUADRATURE or GM_COV_SURROGATE            */
  int32_t deflate;        /* 0 or 64: deflation vectors of the FP32
                             preconditioner (variance panels and mean CG):
                             M^-1 + Y (Theta^-1 - I) Y^T from 64 Ritz pairs of
                             the Jacobi-scaled B, refreshed per posterior
                             update (the paper's PCG solves, App. A.2, with a
                             stronger preconditioner; same results within
                             cg_tol); single-field FP32 contexts, ignored
                             otherwise.  Other values: GM_E_INVAL          */
  double surrogate_gate;  /* surrogate entries whose estimated absolute error
                             after the taper, W K |y - y_true|, exceeds this
                             are recomputed by quadrature (default 1e-4)      */
  double probe_factor;    /* 0: exact marginal variances (one solve per star).
                             > 0: probed variances (Tang & Saad 2012): stars
                             closer than probe_factor x cutoff never share a
                             colour class, each class shares one solve; the
                             error is the neglected cross terms, which decay
                             with the distance (measured 4e-8 relative at
                             2 x cutoff on a 20,000-star 5-degree field)      */
  int32_t quad_rule;      /* GM_QUAD_BAND (default: the converged band rule;
                             n_nodes unused) or GM_QUAD_GL (n_nodes
                             Gauss-Legendre nodes per sightline).  With
                             cov_source = GM_COV_SURROGATE the rule is the
                             surrogate's training target and its fallback  */
  int32_t tc_products;    /* BF16 products per step of the FP32 tensor-core
                             panel product: 6 (default; 0 reads as 6),
                             FP32-grade products from three-piece splits of
                             both operands; or 3 (K1 PD2 + K2 PD1 + K1 PD1,
                             the "mixed" form: half the tensor work, product
                             errors ~1e-5 relative).  Used by FP32 contexts
                             on the tensor-core product, ignored otherwise  */
} gm_config;

/* Device memory hooks.  When given, every device allocation of the context
 * goes through alloc/free (e.g. a framework's caching allocator); when NULL,
 * the library uses cudaMallocAsync/cudaFreeAsync on the context stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} gm_allocator;

/* Counters of the last gm_build_cov / gm_ep_sweep / posterior refresh. */
typedef struct {
  int64_t n_stars;
  int64_t nnz;             /* stored entries of K (both triangles + diagonal) */
  int64_t n_pairs;         /* unique pairs integrated (i <= j)                */
  int64_t cg_iters_mean;   /* CG iterations of the last posterior-mean solve  */
  int64_t cg_iters_var;    /* CG iterations summed over variance panels       */
  int64_t sites_skipped;   /* site updates skipped in the last sweep          */
  int64_t kernel_launches; /* kernels launched by the last API call           */
  double last_max_delta;   /* largest relative site change of the last sweep  */
  double cg_resid_mean;    /* final relative residual of the mean solve       */
  double cg_resid_var;     /* largest final relative residual of a variance   */
  int64_t surrogate_fallback; /* entries recomputed by quadrature (last build) */
  double surrogate_loss;   /* final training loss (last gm_surrogate_train)    */
  double surrogate_val_rmse; /* RMSE of ln K on fresh pairs, tensor-core path  */
  double surrogate_gate_frac; /* fraction of those pairs above the gate
                                (estimated error with the taper applied)    */
  int64_t probe_colours;   /* colour classes (variance solves) when probing,
                              summed over fields (last gm_build_cov)          */
  int64_t tile_ksteps;     /* tensor-core tiles: K-steps of 16 union columns
                              summed over 128-row blocks (0: CUDA-core path)  */
  int64_t variance_panel_width; /* right-hand sides per panel of the last
                              multi-RHS solve (each product launch covers
                              this many columns)                             */
  int64_t tile_variant;    /* tensor-core tile product in use: 0 untuned or
                              CUDA-core path, 1-2 synchronous gathers, 3
                              warp-specialised ring, 4 B operand copied from
                              BF16 planes                                    */
} gm_stats;

/* Fills *cfg with defaults: sigma2 1, L0 20 pc, rho_bar 1e-3 mag/pc, cutoff
 * 3 L0, 32 nodes, lognormal form, Wendland taper, FP64, Gaussian-in-A
 * likelihood, damping 1, cavity floor 1e-8, CG tol 1e-10 / 2000 iterations,
 * automatic panel width, warm-started variance solves, quadrature entries,
 * surrogate gate 1e-3. */
void gm_config_default(gm_config* cfg);

/* Creates a context for n >= 1 stars (Sect. 3: observed (l, b), distance s
 * known, one extinction observation per star, Sect. 4.1 eq. like_factor).
 *   l, b        : Galactic coordinates, radians, length n
 *   s           : distances, pc, > 0, length n
 *   obs         : A_obs (mag) for GM_LIK_GAUSS_IN_A, or ln A_obs for
 *                 GM_LIK_GAUSS_IN_LNA, length n
 *   obs_sigma   : noise standard deviation of obs, > 0, length n
 *   stream      : cudaStream_t to issue work on (NULL = legacy default)
 *   alloc       : device-memory hooks or NULL
 * Sites start at zero (posterior = prior).  Errors: GM_E_INVAL on bad sizes,
 * pointers, non-finite or out-of-range values; GM_E_NOMEM; GM_E_CUDA. */
gm_status gm_ep_init(gm_ctx** out, const gm_config* cfg, int64_t n,
                     const double* l, const double* b, const double* s,
                     const double* obs, const double* obs_sigma, void* stream,
                     const gm_allocator* alloc);

/* Creates a context holding n_fields independent fields (sky fields /
 * sub-catalogues, Sect. 4.1) that are solved together: stars of different
 * fields are never neighbours, so K is block diagonal, and every kernel of
 * the build and of the sweeps runs over all fields in one launch (the
 * variance solves of all fields as one packed multi-panel CG, replayed from
 * a CUDA graph).  Arguments as gm_ep_init, plus
 *   field_id     : field of each star, 0 <= id < n_fields (int32, host or
 *                  device, length n; NULL only when n_fields == 1)
 *   field_L0     : outer scale per field (host, length n_fields; NULL = cfg)
 *   field_cutoff : cutoff per field (host, length n_fields; NULL = cfg)
 * Several fields require GM_PREC_FP32 and the quadrature source, and
 * gm_predict is not available for them (GM_E_STATE). */
gm_status gm_ep_init_fields(gm_ctx** out, const gm_config* cfg, int64_t n, const double* l,
                            const double* b, const double* s, const double* obs,
                            const double* obs_sigma, int32_t n_fields, const int32_t* field_id,
                            const double* field_L0, const double* field_cutoff, void* stream,
                            const gm_allocator* alloc);

/* Assembles K (CSR over the internal order, both triangles, rows sorted) and
 * the prior mean m (Sect. 3): neighbour search within cutoff_pc, sightline
 * double quadrature per unique pair, log1p and taper.  Writes the number of
 * stored entries to *nnz_out (may be NULL).  Must precede gm_ep_sweep and
 * gm_predict.  Reads one scalar back to size the CSR (one stream sync). */
gm_status gm_build_cov(gm_ctx* ctx, int64_t* nnz_out);

/* Runs n_sweeps parallel EP iterations (App. A.2), stopping early when the
 * largest relative site change is below tol (tol <= 0: never early).  Each
 * sweep: posterior mean by PCG on B = I + S^1/2 K S^1/2, marginal variances
 * by multi-RHS PCG, then FP64 cavity / tilted / moment-matched site update
 * for every star.  Outputs (may be NULL): sweeps done, last max change.
 * Errors: GM_E_STATE (no K), GM_E_NOT_SPD, GM_E_NOCONV, GM_E_NONFINITE. */
gm_status gm_ep_sweep(gm_ctx* ctx, int32_t n_sweeps, double tol,
                      int32_t* sweeps_done, double* max_delta);

/* Posterior predictive mean and variance of ln A at nq query points
 * (l, b in radians, s in pc; Sect. 2 eq. cond_GP0 with the sites as
 * observations).  Cross-covariances use the same quadrature, cutoff and
 * taper as K.  mean_out, var_out: length nq, host or device. */
gm_status gm_predict(gm_ctx* ctx, int64_t nq, const double* l, const double* b,
                     const double* s, double* mean_out, double* var_out);

/* Extinction pseudo-density dA/ds (Sect. 5): for each query (l, b, s) the
 * joint posterior predictive of ln A at s and at s + ds on the same sightline
 * (Sect. 2 eq. cond_GP0), and the mean and variance of (A2 - A1) / ds under
 * the paper's condition A2 > A1 (closed-form truncated bivariate-lognormal
 * moments where the paper samples).  ds > 0 (pc; the paper uses 10).
 * Outputs, host or device: mean_out 2 nq (ln A at s, at s + ds per query),
 * cov_out 3 nq (variance at s, variance at s + ds, their covariance),
 * dens_out 2 nq (mean, variance of the pseudo-density, mag/pc).  Single-field
 * contexts; GM_E_INVAL for ds <= 0 or a non-positive distance. */
gm_status gm_predict_pairs(gm_ctx* ctx, int64_t nq, const double* l, const double* b,
                           const double* s, double ds, double* mean_out, double* cov_out,
                           double* dens_out);

/* Joint posterior predictive of ln A at m points of each of nsl sightlines
 * (Sect. 2 eq. cond_GP0 for the points of a sightline together; Sect. 5
 * conditions these joint predictives on dA/ds >= 0).
 * l, b: nsl directions (radians); s: nsl x m distances (pc), strictly
 * increasing along each sightline (row q holds sightline q).  Host or device.
 * mean_out: nsl x m; cov_out: nsl x m x m (row-major per sightline,
 * symmetric).  The prior covariance of two points of one sightline uses the
 * same quadrature (chord 0), cutoff and taper as K.  1 <= m <= 1024.
 * Single-field contexts; GM_E_INVAL for distances that do not increase or are
 * not finite and > 0. */
gm_status gm_predict_sightlines(gm_ctx* ctx, int64_t nsl, int32_t m, const double* l,
                                const double* b, const double* s, double* mean_out,
                                double* cov_out);

/* Samples of each sightline's Gaussian N(mean_q, cov_q) truncated to a
 * non-decreasing sequence a_0 <= a_1 <= ... <= a_{m-1}: the condition
 * dA/ds >= 0 of Sect. 5, by the exact Hamiltonian Monte Carlo of Pakman &
 * Paninski (2014) that the paper uses.  Each step moves for time pi/2 from a
 * fresh momentum and mirrors the velocity at every wall it meets; the chain
 * starts from the running maximum of the mean (point i raised by 1e-9 i).
 * mean: nsl x m; cov: nsl x m x m (the lower triangle is read), e.g. the
 * output of gm_predict_sightlines; momenta: nsl x (n_burn + n_samples) x m
 * standard normal draws (the caller supplies the randomness; step k of
 * sightline q uses momenta[(q (n_burn + n_samples) + k) m ...]).
 * samples_out: nsl x n_samples x m (the steps after the n_burn first);
 * hits_out: nsl wall-hit counts, or NULL.  All host or device.  Needs no K
 * (any context: its stream and allocator).  Errors: GM_E_NONFINITE (a mean
 * or covariance entry not finite; nothing is written), GM_E_NOT_SPD (a covariance not positive
 * definite: that sightline's samples are NaN, the others are written),
 * GM_E_NOCONV (a step met 10,000 walls before its time was used). */
gm_status gm_monotone_sample(gm_ctx* ctx, int64_t nsl, int32_t m, const double* mean,
                             const double* cov, const double* momenta, int32_t n_burn,
                             int32_t n_samples, double* samples_out, int64_t* hits_out);

/* Posterior of the log-extinction u at R inducing points under the paper's
 * partially independent conditional approximation (Sect. 4.1, simplified
 * case; App. B): the stars are split into sub-catalogues that are
 * conditionally independent given u, each with the exact GP conditional
 * a_k | u ~ N(m_k + A_k (u - mu_u), K_kk - A_k K_uk), A_k = K_ku K_uu^-1, and
 * a Gaussian observation of each a_n.  Block-site EP over u reaches its fixed
 * point in one parallel sweep here (every factor is Gaussian), so the result
 * is the PITC posterior:
 *   cov = (K_uu^-1 + sum_k A_k^T C_k^-1 A_k)^-1,
 *   mean = cov (K_uu^-1 mu_u + sum_k A_k^T C_k^-1 (a~_k - m_k + A_k mu_u)),
 * C_k = K_kk - A_k K_uk + diag(sigma_k^2).  K_kk are the stored entries of K
 * (gm_build_cov); K_ku, K_uu and the prior mean mu_u at the inducing points
 * come from the same quadrature, cutoff and taper.
 * block_of: sub-catalogue of each star, caller order, int32 in
 * [0, n_blocks), host or device; at most 8192 stars per sub-catalogue.
 * l, b, s: the R inducing points (radians, pc; 1 <= R <= 4096).
 * mean_out: R; cov_out: R x R row-major; host or device.
 * Needs a single-field FP64 context with GM_LIK_GAUSS_IN_LNA (the stars'
 * observations are then a~ = ln A_obs with standard deviation obs_sigma) and
 * the covariance built (else GM_E_STATE).  GM_E_NOT_SPD when K_uu, a C_k or
 * the posterior precision has no Cholesky factor. */
gm_status gm_pic_posterior(gm_ctx* ctx, int32_t n_blocks, const int32_t* block_of, int64_t R,
                           const double* l, const double* b, const double* s,
                           double* mean_out, double* cov_out);

/* PIC predictive of ln A at nq query points (the paper's partially
 * independent conditional, Sect. 4.1 / App. B), after gm_pic_posterior on
 * the same context (else GM_E_STATE; gm_build_cov discards the posterior).
 * A query assigned to sub-catalogue k depends on the other sub-catalogues
 * only through u: with A_s = k_su K_uu^-1, D = k_sk - K_ku A_s^T, g = C_k^-1 D
 * and L = A_s - g^T A_k,
 *   mean = m_s + g^T (a~_k - m_k) + L (mean_u - mu_u),
 *   var  = k_ss - A_s k_us - g^T D + L cov_u L^T.
 * q_block: sub-catalogue of each query (int32 in [0, n_blocks)); l, b, s the
 * queries (radians, pc); mean_out, var_out: nq.  All host or device. */
gm_status gm_pic_predict(gm_ctx* ctx, int64_t nq, const int32_t* q_block, const double* l,
                         const double* b, const double* s, double* mean_out, double* var_out);

/* Mean function of the extinction pseudo-density (Sect. 5 set-up): an
 * exponential disc plus a Gaussian bump along the line of sight,
 *   rho(x) = rho0 exp(-(R(x) - R_sun)/L - |z|/H) + A_b N(|x|; s_b, w^2),
 * x heliocentric (pc, x_1 towards the Galactic centre, x_3 towards the north
 * Galactic pole), R(x) = |(R_sun - x_1, x_2)|.  The prior mean of ln A_i
 * becomes ln E[A_i] - K_ii/2 with E[A_i] the line integral of rho (disc by a
 * 64-node Gauss-Legendre rule, bump in closed form); the covariance stays
 * that of the stationary relative fluctuations.  Applied to the stars now
 * (if the covariance is built) and by every later gm_build_cov and
 * prediction.  theta = {L, H, rho0, s_b, A_b} (pc, pc, mag/pc, pc, mag), all
 * > 0 (host); r_sun_pc, bump_width_pc > 0.  theta = NULL restores the
 * constant mean density rho_bar.  One-field contexts only (GM_E_STATE). */
gm_status gm_set_mean_fn(gm_ctx* ctx, const double* theta, double r_sun_pc,
                         double bump_width_pc);

/* Learning phase for the five mean-function hyperparameters (Sect. 2, eq.
 * example_learning; Sect. 4.1 simplified case; Sect. 5 log-normal
 * hyperpriors).  Needs likelihood GM_LIK_GAUSS_IN_LNA and the lognormal form
 * (GM_E_INVAL otherwise) and a built covariance (GM_E_STATE).  The marginal
 * likelihood is then exact, atilde ~ N(m(theta), K + Sigma), and the mode of
 * ln p(theta | atilde) in phi = ln theta is found by Newton steps (gradient
 * J^T (K + Sigma)^-1 (atilde - m) - (phi - mu)/s^2 from one posterior-mean
 * solve; Hessian by central differences of the gradient, step 1e-4 in phi,
 * shifted until positive definite; steps halved until the log posterior
 * rises) until the largest step is below tol or max_iter steps.
 *   theta0      : starting point (5 values > 0)
 *   prior_mean, prior_sd : log-normal hyperprior of each parameter, given by
 *                 its mean and standard deviation (natural units; the paper
 *                 takes sd = mean)
 *   theta_out   : the mode (5); cov_out (may be NULL): the Laplace
 *                 covariance of phi = ln theta at the mode (5 x 5 row-major);
 *   log_post_out (may be NULL): -1/2 r^T (K + Sigma)^-1 r + ln p(phi) there
 *                 (the theta-dependent part of the log posterior);
 *   iters_out (may be NULL): Newton steps taken.
 * All host pointers.  On return the context holds the mean function at the
 * mode (as after gm_set_mean_fn), the exact Gaussian sites tau = 1/sigma^2,
 * nu = atilde/sigma^2, and the posterior mean for them; the variances are
 * recomputed by the next call that needs them. */
gm_status gm_learn_mean(gm_ctx* ctx, const double* theta0, const double* prior_mean,
                        const double* prior_sd, double r_sun_pc, double bump_width_pc,
                        int32_t max_iter, double tol, double* theta_out, double* cov_out,
                        double* log_post_out, int32_t* iters_out);

/* Marginal posterior mean and variance of ln A for every star under the
 * current sites (refreshed if the sites changed).  Length n each. */
gm_status gm_get_posterior(gm_ctx* ctx, double* mean_out, double* var_out);

/* Site natural parameters (tau, nu): site_i(a) = exp(-tau a^2/2 + nu a).
 * gm_set_sites restores a saved state (tau >= 0, finite). Length n each. */
gm_status gm_get_sites(gm_ctx* ctx, double* tau_out, double* nu_out);
gm_status gm_set_sites(gm_ctx* ctx, const double* tau, const double* nu);

/* Prior mean m and diagonal K_ii (length n, caller order). */
gm_status gm_get_prior(gm_ctx* ctx, double* mean_out, double* kdiag_out);

/* Internal star order: perm[k] = caller index of internal star k (length n). */
gm_status gm_get_perm(gm_ctx* ctx, int64_t* perm_out);

/* K in CSR over the internal order: row_ptr (n+1), col (nnz, int32),
 * val (nnz, FP64, converted from the stored precision). */
gm_status gm_get_csr(gm_ctx* ctx, int64_t* row_ptr_out, int32_t* col_out,
                     double* val_out);

/* Stored covariance entries K_ij of the log-extinctions (Sect. 3, tapered as
 * used by the solves) for nq caller index pairs (i[q], j[q]); 0 where the
 * pair is beyond the cutoff.
 * i, j: int64, host or device; out: nq doubles, host or device.
 * GM_E_INVAL for an index outside [0, n); GM_E_STATE before gm_build_cov. */
gm_status gm_get_entries(gm_ctx* ctx, int64_t nq, const int64_t* i, const int64_t* j,
                         double* out);

/* Colour class of each star (caller order, int32, length n) when probing is
 * on (probe_factor > 0, after gm_build_cov); classes are numbered from 0 per
 * field; stars closer than probe_factor x cutoff have different classes.
 * These classes share the variance solves of the EP marginals (App. A.2,
 * eq. cavity).  GM_E_STATE if no colouring exists. */
gm_status gm_get_probe_colours(gm_ctx* ctx, int32_t* colour_out);

gm_status gm_get_stats(gm_ctx* ctx, gm_stats* out);

/* The context's cudaStream_t. */
void* gm_stream(gm_ctx* ctx);

/* Per-kernel timing.  gm_profile(ctx, 1) makes every later launch record a
 * CUDA event pair on the context stream; totals per kernel name accumulate
 * until gm_profile(ctx, 0), which also clears them.  gm_kernel_time_count
 * returns the number of distinct kernels timed so far; gm_kernel_time
 * returns the k-th one's name (static string), launch count and summed
 * device time in ms.  Timing adds two event records per launch. */
gm_status gm_profile(gm_ctx* ctx, int32_t enable);
int32_t gm_kernel_time_count(gm_ctx* ctx);
gm_status gm_kernel_time(gm_ctx* ctx, int32_t k, const char** name, int64_t* launches,
                         double* total_ms);

/* Covariance surrogate (no counterpart in the paper, which evaluates every
 * entry by the sightline integral of Sect. 3): an MLP with 5 inputs (the
 * pair's scale-free geometry ln(sqrt(s_i s_j)/L0)/4, |s_i - s_j|/(3 L0),
 * |u_i - u_j| sqrt(s_i s_j)/(3 L0), sigma2 and ln(L0/20 pc)), three
 * hidden layers of 64 SiLU units and 2 outputs: y = ln K (K = log1p(R)
 * before the taper) and e, an estimate of ln |y - y_true|.  It runs on the
 * tensor cores with BF16 operands and FP32 accumulation.
 * Parameters are FP32, gm_surrogate_param_count() of them, laid out as
 * W1[5][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64][2], b4[2]
 * (W[k][n] maps input k to output n). */
int64_t gm_surrogate_param_count(void);
gm_status gm_surrogate_set_params(gm_ctx* ctx, const float* params, int64_t n);
gm_status gm_surrogate_get_params(gm_ctx* ctx, float* params_out, int64_t n);
/* Trains the surrogate of this context's hyperparameters on the GPU: n_pairs
 * pair geometries like those of the covariance (distances spanning the
 * context's stars, separations up to the cutoff) with targets from the
 * sightline quadrature; `steps` Adam steps on mini-batches of `batch` pairs
 * with learning rate lr decaying by cosine to lr/100; FP32 forward and
 * backward kernels.  Starts from the current parameters if set, else from a
 * seeded He initialisation.  Afterwards evaluates the tensor-core network on
 * fresh pairs; results go to gm_stats (surrogate_*). */
gm_status gm_surrogate_train(gm_ctx* ctx, int64_t n_pairs, int32_t steps, int32_t batch,
                             double lr, uint64_t seed);
/* Loss and gradient of the training objective on n given samples (features
 * X[n][5] and targets Y[n] = ln K, FP32, host or device), with error-head
 * weight lam: grad_out has gm_surrogate_param_count() entries (host or
 * device), *loss_out the loss.  For checking the backward pass. */
gm_status gm_surrogate_grad(gm_ctx* ctx, int64_t n, const float* X, const float* Y, double lam,
                            float* grad_out, double* loss_out);
/* Evaluates the surrogate for n pairs given by distances si, sj (pc) and
 * chord |u_i - u_j| (host or device arrays), at sigma2 and L0 (pc).
 * Outputs y and e (FP32, length n).  GM_E_STATE without parameters. */
gm_status gm_surrogate_eval(gm_ctx* ctx, int64_t n, const double* si, const double* sj,
                            const double* chord, double sigma2, double L0, float* y_out,
                            float* e_out);

/* Streamed assembly of a block of covariance rows: for a catalogue whose
 * sparse covariance does not fit in device memory (a million stars within
 * the cutoff of each other by the ten thousand: ~3.7e10 entries), rows are
 * assembled block by block and handed to the caller.  Rows row0 .. row0 +
 * nrows - 1 in the context's internal order (gm_get_perm maps internal to
 * caller indices); each row lists every star within the cutoff (the row's
 * own star included), columns as internal indices in increasing order,
 * values the covariance entries of Sect. 3 with the taper, computed as
 * gm_build_cov would (source GM_COV_QUADRATURE: the context's node rule;
 * GM_COV_SURROGATE: the trained network, with the node rule where the
 * estimated error exceeds the gate and on the diagonal).  No gm_build_cov is
 * needed; one-field contexts only (GM_E_STATE).
 *   capacity     : entries col_out / val_out can hold; if the block has more,
 *                  GM_E_INVAL with *nnz_out set (call again with room)
 *   row_ptr_out  : nrows + 1 offsets (int64), from 0
 *   col_out      : int32 columns; val_out: float (FP32 contexts) or double
 *   nnz_out      : entries of the block; fallback_out (may be NULL): entries
 *                  recomputed by the node rule (diagonal included)
 * Host or device pointers. */
gm_status gm_cov_rows(gm_ctx* ctx, int64_t row0, int64_t nrows, int32_t source,
                      int64_t capacity, int64_t* row_ptr_out, int32_t* col_out, void* val_out,
                      int64_t* nnz_out, int64_t* fallback_out);

/* Allocation-free EP site update.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory while they run --
 * frameworks that own every device allocation through their own pool,
 * processes working inside a fixed, pre-reserved memory budget, and service
 * loops that must not call cudaMalloc/cudaFree on their latency path.  It
 * performs the same parallel EP site update as one gm_ep_sweep (cavity,
 * tilted moments, moment matching, damping, skip rules) on caller-owned
 * arrays, without a context and without allocating anything.
 *   n          : number of stars, 1 <= n <= 1,048,576 (GM_E_INVAL beyond)
 *   mu, var    : posterior marginal mean and variance of ln A per star
 *   obs, obs_sigma : observation and its noise standard deviation
 *   tau, nu    : site parameters, updated in place
 *   likelihood, damping, vc_floor : as in gm_config
 *   stream     : cudaStream_t to run on (NULL = legacy default stream)
 *   max_delta_out, skipped_out : host pointers (may be NULL) receiving the
 *                largest relative site change and the number of skipped stars
 * All arrays must be DEVICE pointers of the current device (or managed
 * memory), length n; host pointers and memory of another GPU: GM_E_INVAL.
 * The scratch is a file-scope device array of about 66 KB that every GPU
 * loading the library keeps until the process exits.  The first call on a
 * device (and the first after a device reset) uploads the Gauss-Hermite rule
 * with a synchronous copy and a device synchronisation, so make that first
 * call before any stream capture.
 * All calls share the array: calls whose work overlaps on the GPU race with
 * one another, so serialise them.  The call synchronises `stream` and
 * returns GM_E_NONFINITE if a non-finite value appeared. */
gm_status gm_site_update_noalloc(int64_t n, const double* mu, const double* var,
                                 const double* obs, const double* obs_sigma, double* tau,
                                 double* nu, int32_t likelihood, double damping,
                                 double vc_floor, void* stream, double* max_delta_out,
                                 int64_t* skipped_out);

const char* gm_status_str(gm_status s);
const char* gm_last_error(gm_ctx* ctx);
void gm_destroy(gm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GMEAD_H */
