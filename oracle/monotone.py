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
"""
from __future__ import annotations

import numpy as np
from scipy import linalg


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


def tmvn_hmc(mu, S, F, g, x0, n_samples, rng, burn=50):
    """Samples of N(mu, S) truncated to F x + g >= 0, starting from a feasible
    x0 (exact HMC of the module docstring)."""
    mu = np.asarray(mu, dtype=np.float64)
    L = linalg.cholesky(np.asarray(S, dtype=np.float64), lower=True)
    W = F @ L                         # constraints in z: W z + c >= 0
    c = F @ mu + g
    z = linalg.solve_triangular(L, np.asarray(x0, dtype=np.float64) - mu, lower=True)
    if np.any(W @ z + c < 0):
        raise ValueError("x0 violates the constraints")
    out = np.empty((n_samples, len(mu)))
    for it in range(burn + n_samples):
        v = rng.standard_normal(len(mu))
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


def monotone_sightline(mu, S, n_samples, rng, burn=50):
    """Samples of the sightline predictive N(mu, S) (points in increasing
    distance) conditioned on a_{j+1} >= a_j."""
    m = len(mu)
    F = np.zeros((m - 1, m))
    F[np.arange(m - 1), np.arange(m - 1)] = -1.0
    F[np.arange(m - 1), np.arange(1, m)] = 1.0
    # feasible start: the running maximum of the mean, nudged upwards
    x0 = np.maximum.accumulate(np.asarray(mu, dtype=np.float64)) + 1e-9 * np.arange(m)
    return tmvn_hmc(mu, S, F, np.zeros(m - 1), x0, n_samples, rng, burn)
