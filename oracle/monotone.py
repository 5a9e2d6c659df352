"""Posterior predictive along a sightline conditioned on dA/ds >= 0
(Sect. 5, "Conditioning on dA/ds >= 0").

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

The predictive of the log-extinction at points s_1 < ... < s_m on one
sightline is multivariate normal N(mu, S); requiring the extinction to grow
with distance truncates it to a_{j+1} - a_j >= 0.  The paper samples the
truncated distribution with the exact Hamiltonian Monte Carlo of Pakman &
Paninski ("Exact Hamiltonian Monte Carlo for truncated multivariate
Gaussians", 2014); this module restates that method:

* whiten: a = mu + L z with S = L L^T, so z ~ N(0, I) truncated to
  F L z + (F mu + g) >= 0 (here F takes consecutive differences, g = 0);
* each step draws a momentum p ~ N(0, I) and moves for time pi/2 along the
  exact trajectory of H = (z.z + p.p)/2, z(t) = z cos t + p sin t;
* when the trajectory meets a constraint wall w^T z + c = 0 (w^T z(t) + c =
  r cos(t - phi) + c with r, phi from w^T z and w^T p), the velocity is
  reflected in the wall, v <- v - 2 (w.v / w.w) w, and the motion continues
  from there for the remaining time.

Every sample satisfies the constraints exactly; the chain leaves the
truncated normal invariant.

`sightline_predictive` gives the N(mu, S) the method starts from: the joint
posterior predictive of the log-extinction at m points of one sightline.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg

from . import gmead_oracle as O


def _first_hit(W, c, z, v, t_left, eps=1e-12):
    """Earliest time in (eps, t_left] at which z cos t + v sin t reaches a wall
    W_j . z + c_j = 0 moving outwards; (t, j) or (None, None)."""
    a = W @ z
    b = W @ v
    r = np.hypot(a, b)
    best_t, best_j = None, None
    for j in range(len(c)):
        if r[j] <= abs(c[j]):   # never reaches the wall
            continue
        phi = np.arctan2(b[j], a[j])
        acos = np.arccos(-c[j] / r[j])
        for root in (phi + acos, phi - acos):
            t = np.mod(root, 2.0 * np.pi)
            if eps < t <= t_left:
                # outwards: the constraint value is decreasing through zero
                deriv = -a[j] * np.sin(t) + b[j] * np.cos(t)
                if deriv < 0 and (best_t is None or t < best_t):
                    best_t, best_j = t, j
    return best_t, best_j


def tmvn_hmc(mu, S, F, g, x0, n_samples, rng, burn=50, momenta=None):
    """Samples of N(mu, S) truncated to F x + g >= 0, starting from a feasible
    x0 (exact HMC of the module docstring).  The momentum of step k is
    rng.standard_normal(d), or momenta[k] when a (burn + n_samples, d) array
    of standard normal draws is given."""
    mu = np.asarray(mu, dtype=np.float64)
    L = linalg.cholesky(np.asarray(S, dtype=np.float64), lower=True)
    W = F @ L                         # constraints in z: W z + c >= 0
    c = F @ mu + g
    z = linalg.solve_triangular(L, np.asarray(x0, dtype=np.float64) - mu, lower=True)
    if np.any(W @ z + c < 0):
        raise ValueError("x0 violates the constraints")
    out = np.empty((n_samples, len(mu)))
    for it in range(burn + n_samples):
        v = rng.standard_normal(len(mu)) if momenta is None else np.array(momenta[it], dtype=np.float64)
        t_left = np.pi / 2
        for _ in range(10000):        # walls met within one step
            t, j = _first_hit(W, c, z, v, t_left)
            if t is None:
                z, v = z * np.cos(t_left) + v * np.sin(t_left), -z * np.sin(t_left) + v * np.cos(t_left)
                break
            z, v = z * np.cos(t) + v * np.sin(t), -z * np.sin(t) + v * np.cos(t)
            w = W[j]
            v = v - 2.0 * (w @ v) / (w @ w) * w
            t_left -= t
        if it >= burn:
            out[it - burn] = mu + L @ z
    return out


def monotone_start(mu):
    """Feasible start for a non-decreasing sequence: the running maximum of
    the mean, each point raised by 1e-9 times its index."""
    mu = np.asarray(mu, dtype=np.float64)
    return np.maximum.accumulate(mu) + 1e-9 * np.arange(len(mu))


def monotone_sightline(mu, S, n_samples, rng, burn=50, momenta=None):
    """Samples of the sightline predictive N(mu, S) (points in increasing
    distance) conditioned on a_{j+1} >= a_j."""
    m = len(mu)
    F = np.zeros((m - 1, m))
    F[np.arange(m - 1), np.arange(m - 1)] = -1.0
    F[np.arange(m - 1), np.arange(1, m)] = 1.0
    return tmvn_hmc(mu, S, F, np.zeros(m - 1), monotone_start(mu), n_samples, rng, burn,
                    momenta)


def sightline_predictive(cat, K, m, tau, nu, l, b, s, form=O.FORM_LOGNORMAL,
                         taper=O.TAPER_WENDLAND, Q=None):
    """Joint posterior predictive of a at the points s[q, 0..M-1] (pc) on the
    sightline (l[q], b[q]) of each q: means (nsl, M) and covariances
    (nsl, M, M).

    The noisy-GP conditional of Sect. 2 (eq. cond_GP0) for the M points of a
    sightline together: mean m_* + k_*^T alpha, covariance
    k_** - k_*^T S^1/2 B^-1 S^1/2 k_*.  The prior covariance of two points of
    one sightline comes from the same sightline quadrature (chord 0), taper
    and cutoff as K, their separation being |s_a - s_b|.
    """
    s = np.atleast_2d(np.asarray(s, dtype=np.float64))
    nsl, M = s.shape
    lq = np.repeat(np.asarray(l, dtype=np.float64), M)
    bq = np.repeat(np.asarray(b, dtype=np.float64), M)
    sq = s.reshape(-1)
    st = np.asarray(cat["s"], dtype=np.float64)
    sigma2, L0 = float(cat["sigma2"]), float(cat["outer_scale_pc"])
    rho_bar, cutoff = float(cat["rho_bar"]), float(cat["cutoff_pc"])
    Q = int(cat["n_nodes"] if Q is None else Q)
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * st[:, None]
    uq = O.unit_vectors(lq, bq)
    xq = uq * sq[:, None]
    n, nq = len(st), len(sq)

    def g(r):
        return O.g_of_r(r, sigma2, L0, form)

    def kq(si, sj, chord2, dist):
        v = O.K_from_R(O.pair_R(si, sj, chord2, g, Q), form)
        if taper == O.TAPER_WENDLAND:
            v = v * O.wendland(dist / cutoff)
        return np.where(dist <= cutoff, v, 0.0)

    kss = O.K_from_R(O.pair_R(sq, sq, np.zeros(nq), g, Q), form)
    # prior covariance of the points of each sightline among themselves
    Kp = np.zeros((nsl, M, M))
    ia, ib = np.triu_indices(M, 1)
    for q in range(nsl):
        sa, sb = s[q, ia], s[q, ib]
        v = kq(sa, sb, np.zeros(len(ia)), np.abs(sb - sa))
        Kp[q, ia, ib] = v
        Kp[q, ib, ia] = v
        Kp[q, np.arange(M), np.arange(M)] = kss[q * M:(q + 1) * M]
    # cross-covariances with the stars
    d = np.sqrt(((xq[:, None, :] - x[None, :, :]) ** 2).sum(axis=2))
    qi, sj = np.nonzero(d <= cutoff)
    Ks = np.zeros((nq, n))
    if len(qi):
        chord2 = ((uq[qi] - u[sj]) ** 2).sum(axis=1)
        Ks[qi, sj] = kq(sq[qi], st[sj], chord2, d[qi, sj])
    if form == O.FORM_LOGNORMAL:
        mq = np.log(rho_bar * sq) - 0.5 * kss
    else:
        mq = np.log(rho_bar * sq) - 0.5 * sigma2
    K = np.asarray(K, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    sqt = np.sqrt(tau)
    B = np.eye(n) + sqt[:, None] * K * sqt[None, :]
    L = linalg.cholesky(B, lower=True)
    bb = nu - tau * m
    y = linalg.cho_solve((L, True), sqt * (K @ bb))
    alpha = bb - sqt * y
    mean = (mq + Ks @ alpha).reshape(nsl, M)
    V = linalg.solve_triangular(L, sqt[:, None] * Ks.T, lower=True)   # n x nq
    cov = np.empty((nsl, M, M))
    for q in range(nsl):
        Vq = V[:, q * M:(q + 1) * M]
        cov[q] = Kp[q] - Vq.T @ Vq
    return mean, cov
