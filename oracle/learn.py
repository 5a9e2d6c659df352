"""FP64 CPU statement of hyperparameter learning for the mean function of
the dust density (Sale & Magorrian 2018, Sect. 2 learning phase and Sect. 5
set-up).

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

Sect. 5 models the mean extinction pseudo-density as an exponential disc plus
a Gaussian bump standing in for a spiral arm, with five hyperparameters: the
disc scale length L, scale height H and pseudo-density at the Sun rho0, and
the bump's distance s_b and total integrated extinction A_b (its width along
the line of sight fixed at 400 pc).  Each gets a log-normal hyperprior whose
standard deviation equals its mean.

Readings (the paper states the parameters, not the formulae):
* mean density at heliocentric position x (pc; x-axis towards the Galactic
  centre, z-axis towards the north Galactic pole):
      rho(x) = rho0 exp(-(R(x) - R_sun) / L - |z| / H)
               + A_b / (w sqrt(2 pi)) exp(-(|x| - s_b)^2 / (2 w^2)),
  R(x) = sqrt((R_sun - x_1)^2 + x_2^2) the Galactocentric radius in the
  plane, R_sun = 8000 pc, w = 400 pc.  Along a sightline the bump term
  integrates to A_b [Phi((s - s_b)/w) - Phi(-s_b/w)].
* mean extinction E[A_i] = int_0^{s_i} rho(t u_i) dt, and the prior mean of
  a_i = ln A_i is its lognormal moment match m_i = ln E[A_i] - K_ii / 2 with
  the covariance K of the stationary relative fluctuations (the constant-
  density covariance of gmead_oracle.build_cov); the hyperparameters enter
  the prior mean only.
* likelihood Gaussian in a (the simplified case of Sect. 4.1), so the
  marginal likelihood is exact: atilde | theta ~ N(m(theta), K + Sigma),
  Sigma = diag(sigma_i^2).  The learning phase (Sect. 2, eq.
  example_learning) seeks p(theta | atilde) ~ N(atilde; m, K + Sigma) p(theta).
* parameters phi = ln theta; the log-normal hyperprior with mean M and
  standard deviation S is N(phi; ln M - s^2/2, s^2) with s^2 = ln(1 + S^2/M^2)
  (= ln 2 for S = M).
* the mode is found by Newton steps on phi: the gradient
  g = J^T (K + Sigma)^-1 r - (phi - mu)/s^2 (J = dm/dphi, r = atilde - m) is
  exact; the Hessian is the central difference of g (step 1e-4 in phi),
  symmetrised, and shifted by d I (d doubling from min 1/s^2) until it is
  positive definite; a step that does not raise the log posterior is
  halved.  The Laplace covariance of phi is the inverse of the Hessian at
  the mode.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, linalg, special

R_SUN = 8000.0
BUMP_W = 400.0
NAMES = ("L", "H", "rho0", "s_bump", "A_bump")
# Sect. 5 hyperprior means (pc, pc, mag/pc, pc, mag); standard deviation = mean
PRIOR_MEAN = np.array([3000.0, 150.0, 0.75e-3, 2000.0, 0.1])


def prior_lognormal(mean=PRIOR_MEAN, sd=None):
    """(mu, s2) of the normal prior on phi = ln theta."""
    mean = np.asarray(mean, dtype=np.float64)
    sd = mean if sd is None else np.asarray(sd, dtype=np.float64)
    s2 = np.log1p((sd / mean) ** 2)
    return np.log(mean) - 0.5 * s2, s2


def density(x, theta, r_sun=R_SUN, w=BUMP_W):
    """Mean extinction pseudo-density (mag/pc) at positions x (..., 3)."""
    L, H, rho0, sb, Ab = theta
    x = np.asarray(x, dtype=np.float64)
    R = np.hypot(r_sun - x[..., 0], x[..., 1])
    disc = rho0 * np.exp(-(R - r_sun) / L - np.abs(x[..., 2]) / H)
    d = np.linalg.norm(x, axis=-1)
    bump = Ab / (w * math.sqrt(2 * math.pi)) * np.exp(-0.5 * ((d - sb) / w) ** 2)
    return disc + bump


_GL_X, _GL_W = np.polynomial.legendre.leggauss(200)


def _disc_terms(u, s, theta, r_sun):
    """The disc integrand and its two shape derivatives at the 200 nodes."""
    L, H, rho0, sb, Ab = theta
    u = np.asarray(u, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    t = 0.5 * s[:, None] * (1.0 + _GL_X[None, :])          # (n, 200)
    dR = np.hypot(r_sun - t * u[:, 0:1], t * u[:, 1:2]) - r_sun
    az = np.abs(t * u[:, 2:3])
    f = rho0 * np.exp(-dR / L - az / H)
    return s, f, dR / L, az / H


def mean_extinction(u, s, theta, r_sun=R_SUN, w=BUMP_W):
    """E[A] = int_0^s rho(t u) dt per star: the disc by a 200-node
    Gauss-Legendre rule on [0, s] (the integrand is smooth in t), the bump in
    closed form (the integral of a normal density)."""
    L, H, rho0, sb, Ab = theta
    s, f, _, _ = _disc_terms(u, s, theta, r_sun)
    disc = 0.5 * s * (f @ _GL_W)
    bump = Ab * (special.ndtr((s - sb) / w) - special.ndtr(-sb / w))
    return disc + bump


def prior_mean(u, s, theta, Kdiag, **kw):
    """m_i = ln E[A_i] - K_ii / 2."""
    return np.log(mean_extinction(u, s, theta, **kw)) - 0.5 * np.asarray(Kdiag)


def jacobian(u, s, theta, Kdiag, r_sun=R_SUN, w=BUMP_W):
    """d m / d phi (n x 5), phi = ln theta: d ln E / d ln theta_k, each the
    derivative of the line integral taken under the integral sign (disc:
    rho (R - R_sun)/L, rho |z|/H and rho for L, H, rho0) or of the bump's
    closed form (s_b, A_b).  K_ii does not depend on theta."""
    L, H, rho0, sb, Ab = theta
    s, f, xl, xh = _disc_terms(u, s, theta, r_sun)
    E = mean_extinction(u, s, theta, r_sun, w)
    a, a0 = (s - sb) / w, -sb / w
    pdf = lambda z: np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    cols = [0.5 * s * ((f * xl) @ _GL_W), 0.5 * s * ((f * xh) @ _GL_W), 0.5 * s * (f @ _GL_W),
            sb * Ab * (pdf(a0) - pdf(a)) / w,
            Ab * (special.ndtr(a) - special.ndtr(a0))]
    return np.stack(cols, axis=1) / E[:, None]


def log_posterior(atil, sig, K, m, phi, mu, s2):
    """ln N(atil; m, K + Sigma) + ln N(phi; mu, s2) (Sect. 2, eq.
    example_learning, up to the evidence)."""
    C = K + np.diag(np.asarray(sig) ** 2)
    cf = linalg.cho_factor(C, lower=True)
    r = np.asarray(atil) - m
    quad = r @ linalg.cho_solve(cf, r)
    logdet = 2.0 * np.log(np.diag(cf[0])).sum()
    lp = -0.5 * (quad + logdet + len(r) * math.log(2 * math.pi))
    lp += -0.5 * np.sum((phi - mu) ** 2 / s2 + np.log(2 * math.pi * s2))
    return float(lp)


def learn_mean(u, s, atil, sig, K, theta0, prior=None, max_iter=50, tol=1e-10, h=1e-4, **kw):
    """MAP of the five mean-function hyperparameters and their Laplace
    covariance (in phi = ln theta).  Returns dict(theta, phi, cov_phi,
    log_post, iters)."""
    mu, s2 = prior_lognormal() if prior is None else prior
    Kd = np.diag(K)
    C = K + np.diag(np.asarray(sig) ** 2)
    cf = linalg.cho_factor(C, lower=True)
    atil = np.asarray(atil, dtype=np.float64)

    def grad(ph):
        th = np.exp(ph)
        m = prior_mean(u, s, th, Kd, **kw)
        J = jacobian(u, s, th, Kd, **kw)
        g = J.T @ linalg.cho_solve(cf, atil - m) - (ph - mu) / s2
        return g, J, m

    def hessian(ph):
        Hm = np.empty((5, 5))
        for k in range(5):
            e = np.zeros(5)
            e[k] = h
            Hm[:, k] = -(grad(ph + e)[0] - grad(ph - e)[0]) / (2 * h)
        Hm = 0.5 * (Hm + Hm.T)
        d = 0.0
        while True:
            try:
                np.linalg.cholesky(Hm + d * np.eye(5))
                return Hm + d * np.eye(5)
            except np.linalg.LinAlgError:
                d = 2 * d if d > 0 else float(np.min(1.0 / s2))

    phi = np.log(np.asarray(theta0, dtype=np.float64))
    g, J, m = grad(phi)
    lp = log_posterior(atil, sig, K, m, phi, mu, s2)
    it = 0
    for it in range(1, max_iter + 1):
        step = np.linalg.solve(hessian(phi), g)
        lam = 1.0
        while True:
            ph_new = phi + lam * step
            m_new = prior_mean(u, s, np.exp(ph_new), Kd, **kw)
            lp_new = log_posterior(atil, sig, K, m_new, ph_new, mu, s2)
            if lp_new >= lp or lam < 1e-6:
                break
            lam *= 0.5
        phi, lp = ph_new, lp_new
        g, J, m = grad(phi)
        if np.max(np.abs(lam * step)) < tol:
            break
    cov = np.linalg.inv(hessian(phi))
    return dict(theta=np.exp(phi), phi=phi, cov_phi=cov, log_post=lp, iters=it, grad=g)
