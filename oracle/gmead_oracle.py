"""FP64 CPU oracle: sparse log-extinction covariance + parallel EP + prediction.

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports, links or runs
this file.  It is the plain, slow, obviously-correct statement of what the
GPU path computes, written from Sale & Magorrian, "Large-scale
three-dimensional Gaussian process extinction mapping" (2018):

* The log-extinction a = ln A is a Gaussian process whose covariance is the
  covariance of the log-density integrated along two sightlines (Sect. 3);
  the density fluctuations follow a Kolmogorov spectrum truncated at the
  energy-injection (outer) scale (Sect. 1).  Reading used here: spectrum
  P(k) ~ (k^2 + k0^2)^(-11/6) with k0 = 1/L0, whose isotropic 3-D transform
  is the von Karman (Matern nu = 1/3) correlation phi below.  The density is
  rho = exp(f), f ~ GP(ln rho_bar - sigma2/2, sigma2*phi); the extinction
  A_i = int_0^{s_i} rho dt has E[A_i] = rho_bar s_i and
  Cov(A_i, A_j) = rho_bar^2 * int int expm1(sigma2 phi(r/L0)) dt dt'.
  The log-extinction moments are matched to these ("lognormal" form):
  K_ij = log1p(I_ij / (s_i s_j)), m_i = ln(rho_bar s_i) - K_ii / 2.
  A first-order "linear" form (g = sigma2 phi, K = I/(s_i s_j),
  m = ln(rho_bar s) - sigma2/2) is kept as an option.
* The double sightline integral uses the same Gauss-Legendre rule on each
  sightline as the GPU (nodes t = s (1 + xi)/2), so that parity measures
  arithmetic, not discretisation.
* Sparsity: pairs whose 3-D star separation exceeds the cutoff c are
  dropped; kept entries are multiplied by a Wendland psi_{3,1} taper
  W(h) = (1-h)^4 (4h+1), h = d/c (positive definite in R^3, so the tapered
  matrix stays positive definite by the Schur product theorem), or by 1
  ("hard" cutoff, which can be indefinite).
* Likelihood per star: either Gaussian in ln A (Sect. 4.1, the per-star
  likelihood of the observed log-extinction) or Gaussian in A, the noise
  model of the synthetic observations (A_obs = A + N(0, sigma_A^2)).
* EP: per-star Gaussian sites t_i(a_i) = exp(-tau_i a_i^2 / 2 + nu_i a_i),
  the parallel schedule of App. A.2 (cavity eq. cavity, tilted eq. tilted,
  moment matching of the KL objective eq. KL1'), damping, a floor on the
  cavity variance (Sect. 5) and a skip of updates that would make a site
  precision negative.
* Posterior and prediction: the noisy-GP conditional (Sect. 2, eq.
  cond_GP0) with the site variances 1/tau as the noise matrix.

Everything here is float64.  Each function cites the passage it follows.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss
from scipy import integrate, linalg, sparse, special
from scipy.spatial import cKDTree

NU = 1.0 / 3.0          # Matern order of the Kolmogorov spectrum (11/6 - 3/2)

LIK_GAUSS_IN_A = 0       # A_obs ~ N(exp(a), sigma^2)
LIK_GAUSS_IN_LNA = 1     # a_obs ~ N(a, sigma^2)

FORM_LOGNORMAL = 0
FORM_LINEAR = 1

TAPER_WENDLAND = 0
TAPER_HARD = 1


# ---------------------------------------------------------------------------
# Covariance of the log-density (Sect. 1 and 3)
# ---------------------------------------------------------------------------
def phi(x):
    """Correlation of the log-density at separation x = r / L0.

    Isotropic 3-D Fourier transform of (k^2 + k0^2)^(-11/6), k0 = 1/L0,
    normalised to phi(0) = 1:  phi(x) = 2^(1-nu)/Gamma(nu) x^nu K_nu(x).
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 0
    xv = x[nz]
    out[nz] = (2.0 ** (1.0 - NU) / special.gamma(NU)) * xv ** NU * special.kv(NU, xv)
    return out


def g_of_r(r, sigma2, L0, form=FORM_LOGNORMAL):
    """Integrand of the sightline double integral at 3-D separation r (pc).

    Lognormal form: Cov(rho, rho')/rho_bar^2 = expm1(sigma2 phi(r/L0)).
    Linear form:    sigma2 phi(r/L0).
    """
    c = sigma2 * phi(np.asarray(r) / L0)
    return np.expm1(c) if form == FORM_LOGNORMAL else c


def gl_rule(Q):
    """Gauss-Legendre rule mapped to [0, 1]: nodes zeta, weights w (sum 1)."""
    xi, om = leggauss(Q)
    return 0.5 * (1.0 + xi), 0.5 * om


def unit_vectors(l, b):
    """Direction to Galactic (l, b) (radians) as a unit 3-vector."""
    l = np.asarray(l, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    cb = np.cos(b)
    return np.stack([cb * np.cos(l), cb * np.sin(l), np.sin(b)], axis=-1)


def pair_R(si, sj, chord2, g, Q):
    """R_ij = I_ij / (s_i s_j) with I_ij = int_0^si int_0^sj g(|t u_i - t' u_j|),
    by the Q-node Gauss-Legendre rule on each sightline.

    si, sj: distances; chord2 = |u_i - u_j|^2 (= 2 - 2 cos theta) for each pair;
    g: callable of the separation r.  The separation is evaluated as
    r^2 = (t - t')^2 + t t' chord2, which equals t^2 + t'^2 - 2 t t' cos theta
    without its cancellation near t = t', theta = 0 (where g has a cusp).
    Returns an array of R values.
    """
    zeta, w = gl_rule(Q)
    si = np.asarray(si, dtype=np.float64)
    sj = np.asarray(sj, dtype=np.float64)
    chord2 = np.asarray(chord2, dtype=np.float64)
    out = np.empty(len(si))
    ww = np.outer(w, w)
    step = max(1, 2_000_000 // (Q * Q))
    for p0 in range(0, len(si), step):
        sl = slice(p0, p0 + step)
        t = si[sl, None] * zeta[None, :]            # (P, Q) nodes on sightline i
        tp = sj[sl, None] * zeta[None, :]           # (P, Q) nodes on sightline j
        r2 = ((t[:, :, None] - tp[:, None, :]) ** 2
              + chord2[sl, None, None] * t[:, :, None] * tp[:, None, :])
        r = np.sqrt(r2)
        out[sl] = np.einsum("pqk,qk->p", g(r), ww)
    return out


def wendland(h):
    """Wendland psi_{3,1}: (1-h)^4 (4h+1) on [0,1], 0 beyond."""
    h = np.asarray(h, dtype=np.float64)
    return np.where(h < 1.0, (1.0 - h) ** 4 * (4.0 * h + 1.0), 0.0)


def K_from_R(R, form):
    return np.log1p(R) if form == FORM_LOGNORMAL else R


# ---------------------------------------------------------------------------
# Sparse covariance assembly
# ---------------------------------------------------------------------------
def neighbour_pairs(x, cutoff):
    """All unordered pairs (i < j) with |x_i - x_j| <= cutoff, sorted."""
    tree = cKDTree(x)
    pairs = tree.query_pairs(cutoff, output_type="ndarray")
    if len(pairs) == 0:
        return np.zeros((0, 2), dtype=np.int64)
    pairs = np.sort(pairs, axis=1)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    pairs = pairs[order]
    # cKDTree uses <= r; recheck with the plain Euclidean formula
    d2 = ((x[pairs[:, 0]] - x[pairs[:, 1]]) ** 2).sum(axis=1)
    return pairs[d2 <= cutoff * cutoff]


def build_cov(cat, form=FORM_LOGNORMAL, taper=TAPER_WENDLAND, Q=None,
              dense=True):
    """Sparse covariance K of the log-extinctions and the prior mean m.

    Returns dict(K=dense ndarray or scipy CSR, m=mean, pairs=(i<j) list,
    diag=K_ii).  Follows Sect. 3 (covariance = density covariance integrated
    along both sightlines) with the readings listed in the module docstring.
    """
    l, b, s = (np.asarray(cat[k], dtype=np.float64) for k in ("l", "b", "s"))
    sigma2, L0 = float(cat["sigma2"]), float(cat["outer_scale_pc"])
    rho_bar, cutoff = float(cat["rho_bar"]), float(cat["cutoff_pc"])
    Q = int(cat["n_nodes"] if Q is None else Q)
    n = len(s)
    u = unit_vectors(l, b)
    x = u * s[:, None]

    def g(r):
        return g_of_r(r, sigma2, L0, form)

    diag = K_from_R(pair_R(s, s, np.zeros(n), g, Q), form)
    pairs = neighbour_pairs(x, cutoff)
    i, j = pairs[:, 0], pairs[:, 1]
    chord2 = ((u[i] - u[j]) ** 2).sum(axis=1)
    Kij = K_from_R(pair_R(s[i], s[j], chord2, g, Q), form)
    if taper == TAPER_WENDLAND:
        d = np.sqrt(((x[i] - x[j]) ** 2).sum(axis=1))
        Kij = Kij * wendland(d / cutoff)
    if form == FORM_LOGNORMAL:
        m = np.log(rho_bar * s) - 0.5 * diag
    else:
        m = np.log(rho_bar * s) - 0.5 * sigma2
    if dense:
        K = np.diag(diag)
        K[i, j] = Kij
        K[j, i] = Kij
    else:
        rows = np.concatenate([np.arange(n), i, j])
        cols = np.concatenate([np.arange(n), j, i])
        vals = np.concatenate([diag, Kij, Kij])
        K = sparse.csr_matrix((vals, (rows, cols)), shape=(n, n))
        K.sort_indices()
    return dict(K=K, m=m, diag=diag, pairs=pairs, Kij=Kij, x=x, u=u)


def csr_structure(n, pairs):
    """Row pointer and sorted column indices of the symmetric pattern
    (diagonal + both triangles of `pairs`)."""
    i, j = pairs[:, 0], pairs[:, 1]
    rows = np.concatenate([np.arange(n), i, j])
    cols = np.concatenate([np.arange(n), j, i])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols


# ---------------------------------------------------------------------------
# Posterior given Gaussian sites (Sect. 2 eq. cond_GP0; App. A.2)
# ---------------------------------------------------------------------------
def posterior(K, m, tau, nu):
    """Marginal posterior mean and variance of a for prior N(m, K) times sites
    exp(-tau a^2/2 + nu a).

    Uses the equivalent regression form of eq. cond_GP0 with noise variances
    1/tau and pseudo-observations nu/tau, computed through
    B = I + S^1/2 K S^1/2 (S = diag tau) so that tau_i = 0 is allowed:
      Sigma = K - K S^1/2 B^-1 S^1/2 K,
      mu    = m + K (b - S^1/2 B^-1 S^1/2 K b),  b = nu - tau m.
    Returns (mu, Sigma_diag, alpha) with alpha such that mu = m + K alpha.
    """
    K = np.asarray(K, dtype=np.float64)
    sq = np.sqrt(tau)
    n = len(m)
    B = np.eye(n) + sq[:, None] * K * sq[None, :]
    L = linalg.cholesky(B, lower=True)
    V = linalg.solve_triangular(L, sq[:, None] * K, lower=True)
    Sdiag = np.diag(K) - (V * V).sum(axis=0)
    b = nu - tau * m
    y = linalg.cho_solve((L, True), sq * (K @ b))
    alpha = b - sq * y
    mu = m + K @ alpha
    return mu, Sdiag, alpha


def gp_regression(K, m, y, noise_var):
    """Plain eq. cond_GP0 at the training points themselves:
    mean m + K (K + N)^-1 (y - m), covariance K - K (K + N)^-1 K."""
    C = K + np.diag(noise_var)
    A = linalg.solve(C, K, assume_a="pos")
    mean = m + A.T @ (y - m)
    cov = K - K @ A
    return mean, np.diag(cov)


# ---------------------------------------------------------------------------
# Tilted moments (App. A.2 eqs. cavity, tilted, KL1')
# ---------------------------------------------------------------------------
GH_NODES = 64


def _log_tilted(a, mu_c, v_c, obs, sig2):
    """Log of N(a; mu_c, v_c) * N(obs; exp(a), sig2) up to constants."""
    ea = np.exp(a)
    return -0.5 * (a - mu_c) ** 2 / v_c - 0.5 * (obs - ea) ** 2 / sig2


def tilted_mode(mu_c, v_c, obs, sig2, max_iter=100):
    """Mode and curvature scale of the Gaussian-in-A tilted density.

    Safeguarded Newton ascent on h(a) = ln N(a; mu_c, v_c) + ln N(obs; e^a, sig2),
    started at the precision-weighted combination of the cavity mean and ln(obs)
    (when obs > 0).  Returns (a_hat, s_hat) with s_hat = (-h''(a_hat))^(-1/2),
    or sqrt(v_c) where h is not concave at the mode.
    """
    if obs > 0:
        aL = math.log(obs)
        vL = sig2 / (obs * obs)
        a = (mu_c / v_c + aL / vL) / (1.0 / v_c + 1.0 / vL)
    else:
        a = mu_c

    def h(a):
        return _log_tilted(a, mu_c, v_c, obs, sig2)

    for _ in range(max_iter):
        ea = math.exp(a)
        gr = -(a - mu_c) / v_c + (obs - ea) * ea / sig2
        H = -1.0 / v_c + (obs * ea - 2.0 * ea * ea) / sig2
        step = -gr / H if H < 0 else gr * v_c
        step = max(-1.0, min(1.0, step))
        h0 = h(a)
        k = 0
        while h(a + step) < h0 and k < 60:
            step *= 0.5
            k += 1
        a += step
        if abs(step) <= 1e-14 * (1.0 + abs(a)):
            break
    ea = math.exp(a)
    H = -1.0 / v_c + (obs * ea - 2.0 * ea * ea) / sig2
    s_hat = 1.0 / math.sqrt(-H) if H < 0 else math.sqrt(v_c)
    return a, s_hat


def tilted_moments_gauss_in_a(mu_c, v_c, obs, sig2, G=GH_NODES):
    """Mean and variance of the tilted distribution N(a; mu_c, v_c) N(obs; e^a, sig2)
    by a G-node Gauss-Hermite rule centred at its mode and scaled by its
    curvature (Laplace point).  Returns (mean, var, log Z) with Z the
    normaliser of the tilted density (eq. KL1', C_l)."""
    a_hat, s_hat = tilted_mode(mu_c, v_c, obs, sig2)
    x, w = hermgauss(G)
    a = a_hat + math.sqrt(2.0) * s_hat * x
    h0 = _log_tilted(a_hat, mu_c, v_c, obs, sig2)
    e = w * np.exp(x * x) * np.exp(_log_tilted(a, mu_c, v_c, obs, sig2) - h0)
    S0 = e.sum()
    mean = (e * a).sum() / S0
    var = (e * (a - mean) ** 2).sum() / S0
    logZ = (h0 + math.log(math.sqrt(2.0) * s_hat * S0)
            - 0.5 * math.log(2 * math.pi * v_c) - 0.5 * math.log(2 * math.pi * sig2))
    return mean, var, logZ


def tilted_moments_adaptive(mu_c, v_c, obs, sig2):
    """Brute-force reference for the Gaussian-in-A tilted moments by adaptive
    quadrature (scipy.integrate.quad) over a wide window around the mode."""
    a_hat, s_hat = tilted_mode(mu_c, v_c, obs, sig2)
    h0 = _log_tilted(a_hat, mu_c, v_c, obs, sig2)
    wide = max(s_hat, math.sqrt(v_c))
    lo = min(a_hat, mu_c) - 40.0 * wide
    hi = max(a_hat, mu_c) + 40.0 * wide

    def f(a, k):
        return (a - a_hat) ** k * math.exp(_log_tilted(a, mu_c, v_c, obs, sig2) - h0)

    opts = dict(points=[a_hat, mu_c], limit=2000, epsabs=0.0, epsrel=1e-13)
    M = [integrate.quad(f, lo, hi, args=(k,), **opts)[0] for k in range(3)]
    mean = a_hat + M[1] / M[0]
    var = M[2] / M[0] - (M[1] / M[0]) ** 2
    return mean, var


def tilted_moments_gauss_in_lna(mu_c, v_c, obs, sig2):
    """Closed form: N(a; mu_c, v_c) N(obs; a, sig2) is Gaussian."""
    v = 1.0 / (1.0 / v_c + 1.0 / sig2)
    return v * (mu_c / v_c + obs / sig2), v


# ---------------------------------------------------------------------------
# Parallel EP (App. A.2) with per-star sites
# ---------------------------------------------------------------------------
def ep_sweep(K, m, obs, obs_sigma, tau, nu, lik=LIK_GAUSS_IN_A, damping=1.0,
             vc_floor=1e-8):
    """One parallel EP iteration.

    1. posterior marginals from the current sites (eq. cond_GP0 form above);
    2. per star: cavity (eq. cavity) tau_c = 1/Sigma_ii - tau_i,
       nu_c = mu_i/Sigma_ii - nu_i, with the cavity variance floored
       (Sect. 5); a star whose cavity precision is not positive is skipped;
    3. tilted moments (eq. tilted) and the moment-matched site (eq. KL1'):
       tau_new = 1/v_hat - tau_c, nu_new = mu_hat/v_hat - nu_c;
    4. damped replacement; an update with tau_new < 0 is skipped.
    Returns (tau, nu, max_delta, n_skipped, mu, Sigma_diag).
    """
    tau = np.array(tau, dtype=np.float64)
    nu = np.array(nu, dtype=np.float64)
    mu, Sd, _ = posterior(K, m, tau, nu)
    n = len(m)
    sig2 = np.asarray(obs_sigma, dtype=np.float64) ** 2
    new_tau, new_nu = tau.copy(), nu.copy()
    skipped = 0
    for i in range(n):
        tc = 1.0 / Sd[i] - tau[i]
        ncv = mu[i] / Sd[i] - nu[i]
        if not (tc > 0) or not np.isfinite(tc):
            skipped += 1
            continue
        mc = ncv / tc
        vc = max(1.0 / tc, vc_floor)
        tc = 1.0 / vc
        ncv = mc / vc
        if lik == LIK_GAUSS_IN_LNA:
            mh, vh = tilted_moments_gauss_in_lna(mc, vc, obs[i], sig2[i])
        else:
            mh, vh, _ = tilted_moments_gauss_in_a(mc, vc, obs[i], sig2[i])
        t_new = 1.0 / vh - tc
        n_new = mh / vh - ncv
        if not (t_new >= 0) or not np.isfinite(n_new):
            skipped += 1
            continue
        new_tau[i] = (1.0 - damping) * tau[i] + damping * t_new
        new_nu[i] = (1.0 - damping) * nu[i] + damping * n_new
    dt = np.abs(new_tau - tau) / (1.0 + np.abs(tau))
    dn = np.abs(new_nu - nu) / (1.0 + np.abs(nu))
    max_delta = float(max(dt.max(initial=0.0), dn.max(initial=0.0)))
    return new_tau, new_nu, max_delta, skipped, mu, Sd


def ep_run(K, m, obs, obs_sigma, lik=LIK_GAUSS_IN_A, max_sweeps=50, tol=1e-10,
           damping=1.0, vc_floor=1e-8, tau0=None, nu0=None):
    """Parallel EP from zero sites (posterior = prior) until the largest
    relative site change falls below tol or max_sweeps is reached."""
    n = len(m)
    tau = np.zeros(n) if tau0 is None else np.array(tau0, dtype=np.float64)
    nu = np.zeros(n) if nu0 is None else np.array(nu0, dtype=np.float64)
    sweeps, delta = 0, float("inf")
    while sweeps < max_sweeps:
        tau, nu, delta, _, _, _ = ep_sweep(K, m, obs, obs_sigma, tau, nu, lik,
                                           damping, vc_floor)
        sweeps += 1
        if delta < tol:
            break
    mu, Sd, alpha = posterior(K, m, tau, nu)
    return dict(tau=tau, nu=nu, mu=mu, var=Sd, alpha=alpha, sweeps=sweeps,
                max_delta=delta)


# ---------------------------------------------------------------------------
# Prediction (Sect. 2 eq. cond_GP0, Sect. 3.1 eq. map_dist)
# ---------------------------------------------------------------------------
def predict(cat, K, m, tau, nu, lq, bq, sq, form=FORM_LOGNORMAL,
            taper=TAPER_WENDLAND, Q=None):
    """Posterior predictive mean and variance of a at query points (lq, bq, sq).

    Cross-covariances k_* use the same sightline quadrature and taper as K
    (pairs beyond the cutoff are zero).  With the sites as noisy observations,
    eq. cond_GP0 gives mean m_* + k_*^T alpha and variance
    k_** - k_*^T S^1/2 B^-1 S^1/2 k_*.
    """
    s = np.asarray(cat["s"], dtype=np.float64)
    sigma2, L0 = float(cat["sigma2"]), float(cat["outer_scale_pc"])
    rho_bar, cutoff = float(cat["rho_bar"]), float(cat["cutoff_pc"])
    Q = int(cat["n_nodes"] if Q is None else Q)
    u = unit_vectors(cat["l"], cat["b"])
    x = u * s[:, None]
    uq = unit_vectors(lq, bq)
    sq = np.asarray(sq, dtype=np.float64)
    xq = uq * sq[:, None]
    nq, n = len(sq), len(s)

    def g(r):
        return g_of_r(r, sigma2, L0, form)

    kss = K_from_R(pair_R(sq, sq, np.zeros(nq), g, Q), form)
    d = np.sqrt(((xq[:, None, :] - x[None, :, :]) ** 2).sum(axis=2))
    qi, sj = np.nonzero(d <= cutoff)
    Ks = np.zeros((nq, n))
    if len(qi):
        chord2 = ((uq[qi] - u[sj]) ** 2).sum(axis=1)
        v = K_from_R(pair_R(sq[qi], s[sj], chord2, g, Q), form)
        if taper == TAPER_WENDLAND:
            v = v * wendland(d[qi, sj] / cutoff)
        Ks[qi, sj] = v
    if form == FORM_LOGNORMAL:
        mq = np.log(rho_bar * sq) - 0.5 * kss
    else:
        mq = np.log(rho_bar * sq) - 0.5 * sigma2
    K = np.asarray(K, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    sqt = np.sqrt(tau)
    B = np.eye(n) + sqt[:, None] * K * sqt[None, :]
    L = linalg.cholesky(B, lower=True)
    b = nu - tau * m
    y = linalg.cho_solve((L, True), sqt * (K @ b))
    alpha = b - sqt * y
    mean = mq + Ks @ alpha
    V = linalg.solve_triangular(L, sqt[:, None] * Ks.T, lower=True)
    var = kss - (V * V).sum(axis=0)
    return mean, var


def posterior_sampled(K, m, tau, nu, idx, tol=1e-12):
    """Posterior mean of every star and marginal variances of the stars idx
    for prior N(m, K) (K a scipy sparse matrix) times the sites, through the
    same regression form as `posterior` with B = I + S^1/2 K S^1/2 solved by
    scipy's conjugate gradient (relative residual tol) instead of a dense
    Cholesky factor: mu = m + K (b - S^1/2 B^-1 S^1/2 K b), b = nu - tau m, and
    Sigma_ii = K_ii - v_i^T B^-1 v_i with v_i = S^1/2 K e_i.  For catalogues
    whose dense covariance does not fit."""
    from scipy.sparse import diags
    from scipy.sparse.linalg import LinearOperator, cg
    tau = np.asarray(tau, dtype=np.float64)
    n = len(tau)
    sq = np.sqrt(tau)
    S = diags(sq)
    Bop = LinearOperator((n, n), matvec=lambda v: v + sq * (K @ (sq * v)), dtype=np.float64)
    dB = 1.0 + tau * K.diagonal()
    M = LinearOperator((n, n), matvec=lambda v: v / dB, dtype=np.float64)

    def solve(rhs):
        x, info = cg(Bop, rhs, rtol=tol, atol=0.0, maxiter=20 * n, M=M)
        if info != 0:
            raise RuntimeError("CG did not converge")
        return x

    b = nu - tau * m
    y = solve(sq * (K @ b))
    mu = m + K @ (b - sq * y)
    var = np.empty(len(idx))
    for k, i in enumerate(idx):
        e = np.zeros(n)
        e[i] = 1.0
        v = S @ (K @ e)
        var[k] = K[i, i] - v @ solve(v)
    return mu, var
