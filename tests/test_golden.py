"""Fixtures under tests/golden: the paper's stated settings and physics
(Kolmogorov turbulence of Sect. 1, the Sect. 5 set-up) pinned against the
oracle, and oracle-written worked examples (tests/golden/make_golden.py) that
the oracle must keep reproducing.  CPU only."""
import os

import numpy as np
import pytest
from scipy import special

import oracle as O
from oracle import density as Dn
from synth import catalogue_subset, make_catalogue

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


def test_kolmogorov_small_scale_law(golden_kv):
    """phi is the correlation of Kolmogorov turbulence: Matern order 1/3 and
    1 - phi ~ r^(2/3) at r << L0 with the Matern coefficient."""
    g = golden_kv("kolmogorov_turbulence.txt")
    nu = g["matern_order"][0]
    assert O.NU == pytest.approx(nu, rel=1e-15)
    assert -2.0 * (nu + 1.5) == pytest.approx(g["spectrum_exponent_3d"][0], rel=1e-15)
    assert 2.0 * nu == pytest.approx(g["structure_function_exponent"][0], rel=1e-15)
    x = np.array([1e-6, 1e-5, 1e-4])
    one_minus = 1.0 - O.phi(x)
    law = special.gamma(1 - nu) / special.gamma(1 + nu) * (x / 2.0) ** (2 * nu)
    np.testing.assert_allclose(one_minus, law, rtol=2e-4)
    slope = np.diff(np.log(one_minus)) / np.diff(np.log(x))
    np.testing.assert_allclose(slope, g["structure_function_exponent"][0], rtol=1e-4)


def test_sect5_setup_is_consistent(golden_kv):
    g = golden_kv("sect5_setup.txt")
    assert g["catalogue_boundaries"][0] * len(g["inducing_distances_kpc"]) == \
        g["inducing_points"][0]
    assert g["pair_offset_pc"][0] > 0


def test_ep_posterior_fixture():
    """The oracle's parallel EP still gives the stored worked example."""
    t = _table("ep_posterior_c1_40.txt")
    n = int(t[:, 1].max()) + 1
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(n))
    cv = O.build_cov(cat)
    for lik in (O.LIK_GAUSS_IN_A, O.LIK_GAUSS_IN_LNA):
        obs = cat["A_obs"] if lik == O.LIK_GAUSS_IN_A else np.log(np.abs(cat["A_obs"]))
        sig = cat["A_sigma"] if lik == O.LIK_GAUSS_IN_A else cat["A_sigma"] / np.abs(cat["A_obs"])
        r = O.ep_run(cv["K"], cv["m"], obs, sig, lik=lik, max_sweeps=5, tol=0.0)
        ref = t[t[:, 0] == lik]
        for col, key in ((2, "tau"), (3, "nu"), (4, "mu"), (5, "var")):
            np.testing.assert_allclose(r[key], ref[:, col], rtol=1e-9, atol=1e-12)
    # a worked-example sanity check that does not depend on the oracle: the
    # posterior variance of ln A cannot exceed the prior variance K_ii
    assert np.all(t[:, 5] > 0) and np.all(t[:, 5] <= np.tile(np.diag(cv["K"]), 2))


def test_tilted_moments_fixture():
    t = _table("tilted_moments.txt")
    for mc, vc, ob, s2, mh, vh, lz, ma, va in t:
        m_, v_, l_ = O.tilted_moments_gauss_in_a(mc, vc, ob, s2)
        assert (m_, v_, l_) == pytest.approx((mh, vh, lz), rel=1e-11, abs=1e-13)
        # the stored rule and adaptive columns agree with each other
        assert mh == pytest.approx(ma, abs=1e-7)
        assert vh == pytest.approx(va, rel=1e-6)


def test_density_moments_fixture():
    t = _table("density_moments.txt")
    for m1, m2, s11, s22, s12, dm, dv in t:
        S = np.array([[s11, s12], [s12, s22]])
        got = Dn.density_moments(np.array([m1, m2]), S, 10.0)
        assert got == pytest.approx((dm, dv), rel=1e-12)
        assert dm > 0 and dv > 0   # A2 > A1 makes the density positive


def test_band_rule_fixture():
    """The oracle's band rule keeps its stored values and node counts; on the
    stored diagonals the 64-node rule differs from it as the 1-D reduction
    says it must (more than 30 % at 1000 pc)."""
    from oracle import band as Bd
    t = _table("band_rule.txt")
    g = lambda r: O.g_of_r(r, 1.0, 20.0)  # noqa: E731
    rule = dict(n=6, h0=1e-3, q=3.0, m0=0.25, K=40.0)
    for si, sj, c2, R, ev, R64 in t:
        got, n = Bd.pair_R_band(si, sj, c2, g, 20.0, **rule)
        assert got[0] == pytest.approx(R, rel=1e-12)
        assert n[0] == int(ev)
    diag1000 = t[(t[:, 0] == 1000.0) & (t[:, 1] == 1000.0)][0]
    assert diag1000[5] / diag1000[3] - 1 > 0.3


def test_hmc_chain_fixture():
    """The oracle's exact-HMC chain for the stored input and momenta, and the
    constraint on every stored sample."""
    from oracle import monotone as Mo
    t = _table("hmc_chain.txt")
    assert np.all(np.diff(t, axis=1) >= 0)
    mu = np.array([-1.0, -1.05, -0.98, -1.02])
    S = 0.03 * np.exp(-np.abs(np.arange(4)[:, None] - np.arange(4)[None, :]) / 2.0) \
        + 1e-4 * np.eye(4)
    mom = np.random.default_rng(20170909).standard_normal((12, 4))
    x = Mo.monotone_sightline(mu, S, 10, None, burn=2, momenta=mom)
    np.testing.assert_allclose(x, t, rtol=0, atol=1e-12)
