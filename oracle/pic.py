"""Block-site EP over inducing points with the PI(T)C approximation
(Sect. 4.1, the simplified case; App. B).

TEST INFRASTRUCTURE ONLY -- the CUDA library never imports or runs this file.

The stars are split into K sub-catalogues (blocks).  With u the log-extinction
at R inducing points, PITC (Snelson & Ghahramani 2007) takes the blocks to be
independent given u:  p(a | u) ~ prod_k p(a_k | u), with the exact GP
conditional of each block,

    a_k | u ~ N(m_k + A_k (u - m_u), K_kk - A_k K_uk),   A_k = K_ku K_uu^-1.

In the simplified case the hyperparameters are fixed and each observed
log-extinction is Gaussian, a~_n | a_n ~ N(a_n, sigma_n^2), so

    a~_k | u ~ N(m_k + A_k (u - m_u), C_k),   C_k = K_kk - A_k K_uk + diag(sigma_k^2),

is a Gaussian factor in u.  EP approximates p(u | a~) by the prior times one
Gaussian site q_k(u) per block: cavity = prior x the other sites; tilted =
cavity x p(a~_k | u); the new site = (moment-matched tilted) / cavity.  With
Gaussian factors the tilted distributions are Gaussian, so the first
parallel sweep already gives the fixed point (each site becomes the block's
exact factor) and EP reproduces the PITC posterior exactly; later sweeps do
not move it.

Prediction (PIC): a star or query in block i depends on the other blocks only
through u,  p(a_* | a~) = int p(a_* | a~_i, u) q(u) du, with
a_* | a~_i, u Gaussian (PITC joint of a_* and a~_i given u), linear in u.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg


def _chol_solve(M, B):
    return linalg.cho_solve(linalg.cho_factor(M, lower=True), B)


def block_factor(Kuu, Kku, Kkk, mu_u, m_k, atil_k, sig2_k):
    """Natural parameters (precision Lam, shift eta) of p(a~_k | u) as a
    Gaussian factor in u: exp(-u^T Lam u / 2 + eta^T u)."""
    A = _chol_solve(Kuu, Kku.T).T                   # K_ku K_uu^-1
    C = Kkk - A @ Kku.T + np.diag(sig2_k)
    Ci_A = _chol_solve(C, A)
    Lam = A.T @ Ci_A
    eta = Ci_A.T @ (atil_k - m_k + A @ mu_u)
    return Lam, eta


def ep_blocks(Kuu, blocks, mu_u, max_sweeps=5):
    """Parallel EP over the block sites (module docstring).  blocks: list of
    dicts with Kku, Kkk, m, atil, sig2.  Returns (posterior mean of u,
    posterior covariance of u, list of site (Lam, eta) per sweep)."""
    R = Kuu.shape[0]
    P0 = linalg.inv(Kuu)                            # prior precision
    h0 = P0 @ mu_u
    K = len(blocks)
    sites = [(np.zeros((R, R)), np.zeros(R)) for _ in range(K)]
    history = []
    for _ in range(max_sweeps):
        Ptot = P0 + sum(L for L, _ in sites)
        htot = h0 + sum(e for _, e in sites)
        new = []
        for k, b in enumerate(blocks):
            # cavity: prior x all sites but k
            Pc = Ptot - sites[k][0]
            hc = htot - sites[k][1]
            # tilted: cavity x p(a~_k | u), Gaussian; its moments
            Lk, ek = block_factor(Kuu, b["Kku"], b["Kkk"], mu_u, b["m"], b["atil"], b["sig2"])
            Pt = Pc + Lk
            Ct = linalg.inv(Pt)
            mt = Ct @ (hc + ek)
            # moment matching: new site = N(mt, Ct) / cavity (natural parameters)
            Ps = linalg.inv(Ct) - Pc
            hs = linalg.solve(Ct, mt) - hc
            new.append((0.5 * (Ps + Ps.T), hs))
        sites = new
        history.append(sites)
    Ptot = P0 + sum(L for L, _ in sites)
    htot = h0 + sum(e for _, e in sites)
    Cu = linalg.inv(Ptot)
    return Cu @ htot, 0.5 * (Cu + Cu.T), history


def pitc_posterior_direct(Kuu, blocks, mu_u):
    """Posterior of u under the PITC model by one linear-Gaussian conditioning
    of all blocks at once (block-diagonal noise), without sites."""
    A = np.vstack([_chol_solve(Kuu, b["Kku"].T).T for b in blocks])
    C = linalg.block_diag(*[b["Kkk"] - _chol_solve(Kuu, b["Kku"].T).T @ b["Kku"].T
                            + np.diag(b["sig2"]) for b in blocks])
    m = np.concatenate([b["m"] for b in blocks])
    y = np.concatenate([b["atil"] for b in blocks])
    S = A @ Kuu @ A.T + C                           # Cov(a~)
    G = _chol_solve(S, A @ Kuu).T                   # Kuu A^T S^-1
    mean = mu_u + G @ (y - m)
    cov = Kuu - G @ A @ Kuu
    return mean, 0.5 * (cov + cov.T)


def pic_predict(Kuu, mu_u, post_mean, post_cov, blk, Ksu, Kss_diag, Ksk, m_s):
    """PIC predictive mean and variance at points of block i (blk: the block's
    Kku, Kkk, m, atil, sig2).  Ksu: points x inducing, Kss_diag: prior
    variances of the points, Ksk: points x block stars, m_s: prior means."""
    As = _chol_solve(Kuu, Ksu.T).T                  # K_su K_uu^-1
    Ak = _chol_solve(Kuu, blk["Kku"].T).T
    Ck = blk["Kkk"] - Ak @ blk["Kku"].T + np.diag(blk["sig2"])
    Dsk = Ksk - As @ blk["Kku"].T                   # Cov(a_s, a~_k | u)
    G = _chol_solve(Ck, Dsk.T).T                    # Dsk Ck^-1
    L = As - G @ Ak                                 # coefficient of (u - mu_u)
    mean = m_s + G @ (blk["atil"] - blk["m"]) + L @ (post_mean - mu_u)
    var = (Kss_diag - np.einsum("ij,ij->i", As, Ksu) - np.einsum("ij,ij->i", G, Dsk)
           + np.einsum("ij,jk,ik->i", L, post_cov, L))
    return mean, var
