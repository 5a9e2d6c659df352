"""Probing estimate of the EP posterior marginal variances.

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

The EP cavities need the marginal variances Sigma_ii of the posterior
(App. A.2, eq. cavity).  With B = I + S^1/2 K S^1/2 (S = diag tau) they are

    Sigma_ii = K_ii - v_i^T B^-1 v_i,   v_i = S^1/2 K e_i          (v form)
    Sigma_ii = (1 - (B^-1)_ii) / tau_i                             (unit form)

the unit form being used where the star's own site dominates
(tau_i K_ii >= 1).  Computing them exactly takes one solve with B per star.
Probing (Tang & Saad 2012, "A probing method for computing the diagonal of a
matrix inverse") shares one solve among all stars of a colour class whose
members are farther apart than a distance D: with z_c = sum of the class's
right-hand sides (v_i or e_i) and w_c = B^-1 z_c,

    Sigma_ii ~ K_ii - v_i^T w_c      or      (1 - (w_c)_i) / tau_i.

The error is the sum of the cross terms v_i^T B^-1 v_j (or their unit
analogues) over the other members j of i's class; B^-1 decays with the
separation of the stars, so the error falls quickly as D grows.  A colouring
in which every star has its own colour gives the exact variances.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg
from scipy.spatial import cKDTree


def greedy_colouring(x, D, order=None):
    """Sequential greedy colouring of the graph "|x_i - x_j| < D": each star,
    in `order` (default: index order), takes the smallest colour not held by
    an already coloured star closer than D.  Returns int array of colours."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    order = np.arange(n) if order is None else np.asarray(order)
    colour = -np.ones(n, dtype=np.int64)
    if D <= 0:
        colour[:] = 0
        return colour
    nb = cKDTree(x).query_ball_point(x, np.nextafter(D, 0.0))   # open ball: d < D
    for i in order:
        used = {colour[j] for j in nb[i] if colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def unit_form(K, tau):
    """Stars whose variance uses the unit right-hand side (tau_i K_ii >= 1)."""
    return np.asarray(tau) * np.diag(np.asarray(K)) >= 1.0


def probed_variances(K, tau, colour):
    """Sigma_ii by probing with the given colour classes (dense B, Cholesky
    solves; module docstring for the formulas)."""
    K = np.asarray(K, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    n = len(tau)
    sq = np.sqrt(tau)
    B = np.eye(n) + sq[:, None] * K * sq[None, :]
    cf = linalg.cho_factor(B, lower=True)
    unit = unit_form(K, tau)
    V = sq[:, None] * K                 # column i is v_i
    var = np.empty(n)
    for c in np.unique(colour):
        members = np.flatnonzero(colour == c)
        z = np.zeros(n)
        for i in members:
            if unit[i]:
                z[i] += 1.0
            else:
                z += V[:, i]
        w = linalg.cho_solve(cf, z)
        for i in members:
            var[i] = (1.0 - w[i]) / tau[i] if unit[i] else K[i, i] - V[:, i] @ w
    return var
