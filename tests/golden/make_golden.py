"""Writes the oracle-derived fixtures of this folder.

Calls only the oracle (`oracle/`) and the seeded input generator (`synth/`);
nothing here comes from the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py

Each file starts with '#' lines that give the passage it follows and the
inputs; the numbers are what the oracle computed when the file was written.
`tests/test_golden.py` checks that the oracle still reproduces them, so a
change to the oracle's arithmetic shows up as a failing fixture.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle import band as Bd  # noqa: E402
from oracle import density as Dn  # noqa: E402
from oracle import monotone as Mo  # noqa: E402
from synth import catalogue_subset, make_catalogue  # noqa: E402

N_EP = 40
SWEEPS = 5
TILTED_CASES = [  # (cavity mean, cavity variance, observed A, noise variance)
    (-0.7, 0.30, 0.50, 0.0025),
    (0.2, 1.00, 1.30, 0.0100),
    (-2.0, 0.05, 0.14, 0.0009),
    (0.0, 4.00, -0.05, 0.0025),   # an observation below zero (admitted)
    (1.1, 0.50, 2.80, 0.0400),
]
DENSITY_CASES = [  # (mu1, mu2, S11, S22, S12), pair offset 10 pc
    (-0.50, -0.48, 0.040, 0.042, 0.039),
    (-1.00, -1.05, 0.040, 0.050, 0.030),
    (0.20, 0.21, 0.010, 0.011, 0.0095),
    (-2.30, -2.20, 0.300, 0.310, 0.280),
]


def _header(f, lines):
    for ln in lines:
        f.write("# " + ln + "\n")


def ep_posterior():
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(N_EP))
    cv = O.build_cov(cat)
    rows = []
    for lik in (O.LIK_GAUSS_IN_A, O.LIK_GAUSS_IN_LNA):
        obs = cat["A_obs"] if lik == O.LIK_GAUSS_IN_A else np.log(np.abs(cat["A_obs"]))
        sig = cat["A_sigma"] if lik == O.LIK_GAUSS_IN_A else cat["A_sigma"] / np.abs(cat["A_obs"])
        r = O.ep_run(cv["K"], cv["m"], obs, sig, lik=lik, max_sweeps=SWEEPS, tol=0.0)
        for i in range(N_EP):
            rows.append((lik, i, r["tau"][i], r["nu"][i], r["mu"][i], r["var"][i]))
    path = os.path.join(HERE, "ep_posterior_c1_40.txt")
    with open(path, "w") as f:
        _header(f, [
            "Parallel EP (App. A.2: cavity, tilted moments, moment matching) from zero",
            "sites, %d sweeps, damping 1, on the first %d stars of the 400-star" % (SWEEPS, N_EP),
            "workload (truth = rho_bar s), tapered lognormal covariance of Sect. 3.",
            "lik 0: A_obs ~ N(exp(a), sigma^2) (Sect. 4.1); lik 1: ln|A_obs| ~ N(a, (sigma/|A_obs|)^2).",
            "Written by tests/golden/make_golden.py from oracle/.",
            "columns: lik star tau nu mean_lnA var_lnA",
        ])
        for r in rows:
            f.write("%d %d %.17e %.17e %.17e %.17e\n" % r)


def tilted_moments():
    path = os.path.join(HERE, "tilted_moments.txt")
    with open(path, "w") as f:
        _header(f, [
            "Tilted distribution N(a; mu_c, v_c) N(A_obs; exp(a), sig2) (App. A.2 eq. tilted,",
            "likelihood of Sect. 4.1): log normaliser, mean and variance by the 64-node",
            "Gauss-Hermite rule at the tilted mode; mean and variance by adaptive quadrature.",
            "Written by tests/golden/make_golden.py from oracle/.",
            "columns: mu_c v_c A_obs sig2 | rule: mean var logZ | adaptive: mean var",
        ])
        for mc, vc, ob, s2 in TILTED_CASES:
            mh, vh, lz = O.tilted_moments_gauss_in_a(mc, vc, ob, s2)
            ma, va = O.tilted_moments_adaptive(mc, vc, ob, s2)
            f.write(" ".join("%.17e" % v for v in (mc, vc, ob, s2, mh, vh, lz, ma, va)) + "\n")


def density_moments():
    path = os.path.join(HERE, "density_moments.txt")
    with open(path, "w") as f:
        _header(f, [
            "Pseudo-density (A2 - A1)/ds given A2 > A1 for (a1, a2) ~ N(mu, S), A = exp(a),",
            "ds = 10 pc (Sect. 5), closed-form moments of oracle/density.py.",
            "Written by tests/golden/make_golden.py from oracle/.",
            "columns: mu1 mu2 S11 S22 S12 | density mean (mag/pc) | density variance",
        ])
        for m1, m2, s11, s22, s12 in DENSITY_CASES:
            S = np.array([[s11, s12], [s12, s22]])
            dm, dv = Dn.density_moments(np.array([m1, m2]), S, 10.0)
            f.write(" ".join("%.17e" % v for v in (m1, m2, s11, s22, s12, dm, dv)) + "\n")


BAND_CASES = [  # (si, sj, chord^2) in pc, outer scale 20 pc, sigma2 1
    (40.0, 40.0, 0.0), (1000.0, 1000.0, 0.0), (3000.0, 2950.0, 0.0), (100.0, 120.0, 0.04),
    (1000.0, 1020.0, 1e-4), (500.0, 480.0, 0.0064),
]
BAND_RULE = dict(n=6, h0=1e-3, q=3.0, m0=0.25, K=40.0)


def band_rule():
    path = os.path.join(HERE, "band_rule.txt")
    g = lambda r: O.g_of_r(r, 1.0, 20.0)  # noqa: E731
    with open(path, "w") as f:
        _header(f, [
            "Sightline double integral R = I / (si sj) of Sect. 3 (lognormal form, sigma2 1,",
            "outer scale 20 pc) by the band rule of oracle/band.py with 6 nodes per panel,",
            "first width 1e-3 L0, ratio 3, first m-panel L0/(4c), truncation 40 L0, and by",
            "the 64-node Gauss-Legendre rule.",
            "Written by tests/golden/make_golden.py from oracle/.",
            "columns: si sj chord2 | band R | evaluations | GL64 R",
        ])
        for si, sj, c2 in BAND_CASES:
            R, ev = Bd.pair_R_band(si, sj, c2, g, 20.0, **BAND_RULE)
            R64 = O.pair_R(np.array([si]), np.array([sj]), np.array([c2]), g, 64)[0]
            f.write("%.17e %.17e %.17e %.17e %d %.17e\n" % (si, sj, c2, R[0], ev[0], R64))


def hmc_chain():
    path = os.path.join(HERE, "hmc_chain.txt")
    mu = np.array([-1.0, -1.05, -0.98, -1.02])
    S = 0.03 * np.exp(-np.abs(np.arange(4)[:, None] - np.arange(4)[None, :]) / 2.0) \
        + 1e-4 * np.eye(4)
    mom = np.random.default_rng(20170909).standard_normal((12, 4))
    x = Mo.monotone_sightline(mu, S, 10, None, burn=2, momenta=mom)
    with open(path, "w") as f:
        _header(f, [
            "Exact HMC for a Gaussian truncated to a non-decreasing sequence (the dA/ds >= 0",
            "conditioning of Sect. 5; Pakman & Paninski 2014), oracle/monotone.py:",
            "mu = (-1, -1.05, -0.98, -1.02), S_ij = 0.03 exp(-|i - j| / 2) + 1e-4 delta_ij,",
            "momenta = numpy default_rng(20170909).standard_normal((12, 4)), 2 burn-in steps.",
            "Written by tests/golden/make_golden.py from oracle/.",
            "rows: the 10 samples (4 points each)",
        ])
        for row in x:
            f.write(" ".join("%.17e" % v for v in row) + "\n")


if __name__ == "__main__":
    ep_posterior()
    tilted_moments()
    density_moments()
    band_rule()
    hmc_chain()
