"""Extinction pseudo-density from pairs of posterior-predictive points.

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

Sect. 5 maps the extinction pseudo-density rho kappa = dA/ds: at each grid
point it takes the joint posterior predictive of the log-extinction at the
point and at a second point on the same sightline a distance ds further
away, and the density is the difference of the two extinctions over ds,
with the condition that the farther extinction is the larger one.  The paper
samples that conditional; here its first two moments are written in closed
form.  With (a1, a2) jointly normal (means mu, covariance S) and A = exp(a),
the condition A2 > A1 is a2 > a1, i.e. D = a2 - a1 > 0, and for any linear
combination X = c^T a,

    E[exp(X) 1{D > 0}] = exp(E X + Var X / 2) Phi((E D + Cov(X, D)) / sd(D)),

(complete the square in the bivariate normal integral), so

    E[A2 - A1 | D > 0]       = (E[e^a2 1] - E[e^a1 1]) / P(D > 0)
    E[(A2 - A1)^2 | D > 0]   = (E[e^2a2 1] - 2 E[e^(a1+a2) 1] + E[e^2a1 1]) / P(D > 0),

with P(D > 0) = Phi(E D / sd(D)).  Dividing by ds gives the moments of the
pseudo-density.  The joint predictive of the two points is the noisy-GP
conditional of Sect. 2 (eq. cond_GP0), as for single points in
`gmead_oracle.predict`, with the two points' own covariance entry from the
same sightline quadrature.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg
from scipy.special import ndtr

from . import gmead_oracle as O


def truncated_exp_moment(mu, S, c, cd):
    """E[exp(c^T a) 1{cd^T a > 0}] for a ~ N(mu, S) (2-vectors, 2x2)."""
    mx = c @ mu
    vx = c @ S @ c
    md = cd @ mu
    vd = cd @ S @ cd
    cxd = c @ S @ cd
    return np.exp(mx + 0.5 * vx) * ndtr((md + cxd) / np.sqrt(vd))


def density_moments(mu, S, ds):
    """Mean and variance of (A2 - A1) / ds given A2 > A1, A = exp(a),
    a ~ N(mu, S) (bivariate); closed form of the module docstring."""
    mu = np.asarray(mu, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    cd = np.array([-1.0, 1.0])
    pd = ndtr((cd @ mu) / np.sqrt(cd @ S @ cd))
    e1 = truncated_exp_moment(mu, S, np.array([1.0, 0.0]), cd)
    e2 = truncated_exp_moment(mu, S, np.array([0.0, 1.0]), cd)
    e11 = truncated_exp_moment(mu, S, np.array([2.0, 0.0]), cd)
    e22 = truncated_exp_moment(mu, S, np.array([0.0, 2.0]), cd)
    e12 = truncated_exp_moment(mu, S, np.array([1.0, 1.0]), cd)
    m1 = (e2 - e1) / pd
    m2 = (e22 - 2.0 * e12 + e11) / pd
    return m1 / ds, (m2 - m1 * m1) / (ds * ds)


def predict_pairs(cat, K, m, tau, nu, lq, bq, sq, ds, form=O.FORM_LOGNORMAL,
                  taper=O.TAPER_WENDLAND, Q=None):
    """Joint posterior predictive of a at (l, b, s) and (l, b, s + ds) for each
    query: returns means (nq, 2) and covariances (nq, 2, 2)."""
    lq, bq, sq = (np.asarray(v, dtype=np.float64) for v in (lq, bq, sq))
    nq = len(sq)
    l2 = np.concatenate([lq, lq])
    b2 = np.concatenate([bq, bq])
    s2 = np.concatenate([sq, sq + ds])
    # marginals of all 2 nq points, and the cross terms from the same pieces
    s = np.asarray(cat["s"], dtype=np.float64)
    sigma2, L0 = float(cat["sigma2"]), float(cat["outer_scale_pc"])
    rho_bar, cutoff = float(cat["rho_bar"]), float(cat["cutoff_pc"])
    Q = int(cat["n_nodes"] if Q is None else Q)
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * s[:, None]
    uq = O.unit_vectors(l2, b2)
    xq = uq * s2[:, None]
    n = len(s)

    def g(r):
        return O.g_of_r(r, sigma2, L0, form)

    def kq(si, sj, chord2, dist):
        v = O.K_from_R(O.pair_R(si, sj, chord2, g, Q), form)
        if taper == O.TAPER_WENDLAND:
            v = v * O.wendland(dist / cutoff)
        return np.where(dist <= cutoff, v, 0.0)

    kss = O.K_from_R(O.pair_R(s2, s2, np.zeros(2 * nq), g, Q), form)
    # cross-covariance of the two points of each pair (same sightline)
    k12 = kq(sq, sq + ds, np.zeros(nq), np.full(nq, float(ds)))
    d = np.sqrt(((xq[:, None, :] - x[None, :, :]) ** 2).sum(axis=2))
    qi, sj = np.nonzero(d <= cutoff)
    Ks = np.zeros((2 * nq, n))
    if len(qi):
        chord2 = ((uq[qi] - u[sj]) ** 2).sum(axis=1)
        Ks[qi, sj] = kq(s2[qi], s[sj], chord2, d[qi, sj])
    if form == O.FORM_LOGNORMAL:
        mq = np.log(rho_bar * s2) - 0.5 * kss
    else:
        mq = np.log(rho_bar * s2) - 0.5 * sigma2
    K = np.asarray(K, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    sqt = np.sqrt(tau)
    B = np.eye(n) + sqt[:, None] * K * sqt[None, :]
    L = linalg.cholesky(B, lower=True)
    b = nu - tau * m
    y = linalg.cho_solve((L, True), sqt * (K @ b))
    alpha = b - sqt * y
    mean = mq + Ks @ alpha
    V = linalg.solve_triangular(L, sqt[:, None] * Ks.T, lower=True)   # n x 2nq
    C = V.T @ V                                                        # v^T B^-1 v
    mu = np.stack([mean[:nq], mean[nq:]], axis=1)
    cov = np.empty((nq, 2, 2))
    idx = np.arange(nq)
    cov[:, 0, 0] = kss[:nq] - C[idx, idx]
    cov[:, 1, 1] = kss[nq:] - C[nq + idx, nq + idx]
    cov[:, 0, 1] = cov[:, 1, 0] = k12 - C[idx, nq + idx]
    return mu, cov
