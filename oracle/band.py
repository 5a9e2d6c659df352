"""Converged sightline double integral: a band rule in difference / mean
coordinates (Sect. 3's covariance of the log-extinctions, computed without
the discretisation error of a global Gauss-Legendre rule).

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

The covariance of two stars' extinctions is the density covariance
integrated along both sightlines (Sect. 3):

    I_ij = int_0^si int_0^sj g(|t u_i - t' u_j|) dt' dt,
    |t u_i - t' u_j|^2 = (t - t')^2 + t t' c^2,   c^2 = |u_i - u_j|^2.

The integrand is concentrated where the two points are within a few outer
scales L0 of each other: near the diagonal t = t', and, when the sightlines
diverge (c > 0), near the observer.  A global Q-node Gauss-Legendre rule on
[0, s] spaces its nodes s / Q apart, which for s >> L0 cannot resolve a
kernel of width L0 (at Q = 64, s = 3000 pc, L0 = 20 pc the diagonal comes out
175 % too large).  With d = t - t' and m = (t + t') / 2 (unit Jacobian),

    t t' = m^2 - d^2 / 4,   r^2 = d^2 (1 - c^2 / 4) + m^2 c^2,
    I_ij = int_{-sj}^{si} dd int_{|d|/2}^{min(si - d/2, sj + d/2)} g(r) dm.

The rule:
  * d: breakpoints 0, +-h0 L0, +-h0 L0 (1 + q), +-h0 L0 (1 + q + q^2), ...
    (geometric grading towards the cusp of g at r = 0 on the diagonal),
    truncated at si (positive side) and sj (negative side) or at K L0,
    plus the kink d = si - sj of the inner interval; n-point Gauss-Legendre
    on each panel;
  * m, for c > 0: breakpoints from the lower end with widths
    m0 (L0 / c) q^k up to the upper end or K L0 / c beyond the lower end
    (the integrand decays on the scale L0 / c); n-point Gauss-Legendre on
    each panel.  For c = 0 the integrand does not depend on m and the inner
    integral is (upper - lower) g(|d|) exactly.

The truncation at K L0 drops separations where g < 2e-18 sigma2 for K = 40.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss

DEFAULT = dict(n=8, h0=1e-3, q=2.0, m0=0.25, K=40.0)


def _gl01(n):
    x, w = leggauss(n)
    return 0.5 * (1.0 + x), 0.5 * w


def _graded(a, end, h0, q):
    """Breakpoints a, a + h0, a + h0 (1 + q), ... clipped at end (> a)."""
    out = [a]
    h = h0
    while out[-1] < end:
        out.append(min(end, out[-1] + h))
        h *= q
    return out


def band_nodes(si, sj, chord2, L0, n=8, h0=1e-3, q=2.0, m0=0.25, K=40.0):
    """Nodes (d, m) and weights of the band rule for one pair."""
    c = math.sqrt(chord2)
    z, w = _gl01(n)
    Dp, Dn = min(si, K * L0), min(sj, K * L0)
    br = set(_graded(0.0, Dp, h0 * L0, q)) | {-x for x in _graded(0.0, Dn, h0 * L0, q)}
    if -Dn < si - sj < Dp:
        br.add(si - sj)
    br = sorted(br)
    D, M, W = [], [], []
    for a, b in zip(br[:-1], br[1:]):
        for dk, wk in zip(a + (b - a) * z, (b - a) * w):
            lo = abs(dk) / 2.0
            hi = min(si - dk / 2.0, sj + dk / 2.0)
            if hi <= lo:
                continue
            if c > 0.0:
                sc = L0 / c
                mb = _graded(lo, min(hi, lo + K * sc), m0 * sc, q)
                for ma, mc in zip(mb[:-1], mb[1:]):
                    D.append(np.full(n, dk))
                    M.append(ma + (mc - ma) * z)
                    W.append(wk * (mc - ma) * w)
            else:
                D.append(np.array([dk]))
                M.append(np.array([0.0]))
                W.append(np.array([wk * (hi - lo)]))
    return np.concatenate(D), np.concatenate(M), np.concatenate(W)


def pair_R_band(si, sj, chord2, g, L0, **rule):
    """R_ij = I_ij / (si sj) by the band rule (module docstring) for arrays
    of pairs; g: callable of the separation r.  Also returns the number of
    integrand evaluations of each pair."""
    prm = dict(DEFAULT, **rule)
    si, sj, chord2 = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (si, sj, chord2))
    out = np.empty(len(si))
    evals = np.empty(len(si), dtype=np.int64)
    for p in range(len(si)):
        d, m, w = band_nodes(si[p], sj[p], chord2[p], L0, **prm)
        r = np.sqrt(d * d * (1.0 - chord2[p] / 4.0) + m * m * chord2[p])
        out[p] = (w * g(r)).sum() / (si[p] * sj[p])
        evals[p] = len(w)
    return out, evals


def build_cov_band(cat, form=None, taper=None, **rule):
    """The covariance assembly of `gmead_oracle.build_cov` (same neighbours,
    cutoff, taper and lognormal moment match) with every pair integral, the
    diagonal included, from the band rule.  Returns dict(K (dense), m,
    diag, evals)."""
    from . import gmead_oracle as O
    form = O.FORM_LOGNORMAL if form is None else form
    taper = O.TAPER_WENDLAND if taper is None else taper
    s = np.asarray(cat["s"], dtype=np.float64)
    sigma2, L0 = float(cat["sigma2"]), float(cat["outer_scale_pc"])
    rho_bar, cutoff = float(cat["rho_bar"]), float(cat["cutoff_pc"])
    n = len(s)
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * s[:, None]

    def g(r):
        return O.g_of_r(r, sigma2, L0, form)

    Rd, ed = pair_R_band(s, s, np.zeros(n), g, L0, **rule)
    diag = O.K_from_R(Rd, form)
    pairs = O.neighbour_pairs(x, cutoff)
    i, j = pairs[:, 0], pairs[:, 1]
    chord2 = ((u[i] - u[j]) ** 2).sum(axis=1)
    Rij, ep = pair_R_band(s[i], s[j], chord2, g, L0, **rule)
    Kij = O.K_from_R(Rij, form)
    if taper == O.TAPER_WENDLAND:
        Kij = Kij * O.wendland(np.sqrt(((x[i] - x[j]) ** 2).sum(axis=1)) / cutoff)
    m = np.log(rho_bar * s) - (0.5 * diag if form == O.FORM_LOGNORMAL else 0.5 * sigma2)
    K = np.diag(diag)
    K[i, j] = Kij
    K[j, i] = Kij
    return dict(K=K, m=m, diag=diag, evals=np.concatenate([ed, ep]))
