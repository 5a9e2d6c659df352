"""Pins of the CPU oracle to things other than itself (closed forms, brute
force, independent library routines, limits).  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, linalg

import oracle as O
from synth import catalogue_subset, make_catalogue


# ---------------------------------------------------------------- covariance
def _spectrum(k):
    # Kolmogorov spectrum truncated at the outer scale, L0 = 1 (k0 = 1/L0)
    return (k * k + 1.0) ** (-11.0 / 6.0)


@pytest.mark.parametrize("x", [0.02, 0.1, 0.3, 1.0, 2.0, 4.0, 8.0])
def test_phi_is_fourier_transform_of_truncated_kolmogorov(x):
    """phi(r/L0) equals C(r)/C(0) with C the isotropic 3-D transform of
    P(k) = (k^2 + k0^2)^(-11/6), computed by oscillatory quadrature."""
    den = integrate.quad(lambda k: k * k * _spectrum(k), 0, np.inf,
                         epsabs=0, epsrel=1e-13, limit=500)[0]
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            num = integrate.quad(lambda k: k * _spectrum(k), 0, np.inf,
                                 weight="sin", wvar=x, epsabs=1e-15,
                                 limlst=200)[0] / x
    assert O.phi(np.array([x]))[0] == pytest.approx(num / den, rel=1e-10)


def test_phi_limits():
    assert O.phi(np.array([0.0]))[0] == 1.0
    x = np.linspace(1e-6, 30, 2000)
    p = O.phi(x)
    assert np.all(np.diff(p) < 0) and p[-1] < 1e-11 and p[0] < 1.0


def test_gl_rule_exact_on_quadratic_in_r2():
    """g(r) = r^2 and r^4 are polynomials of degree <= 4 in (t, t'); the rule
    must reproduce the closed-form sightline averages exactly."""
    rng = np.random.default_rng(1)
    si, sj = rng.uniform(50, 3000, 20), rng.uniform(50, 3000, 20)
    c = np.cos(rng.uniform(0, 0.2, 20))
    R2 = O.pair_R(si, sj, 2 - 2 * c, lambda r: r ** 2, 8)
    ref2 = (si ** 2 + sj ** 2) / 3.0 - c * si * sj / 2.0
    np.testing.assert_allclose(R2, ref2, rtol=1e-12)
    R4 = O.pair_R(si, sj, 2 - 2 * c, lambda r: r ** 4, 8)
    ref4 = (si ** 4 / 5 + sj ** 4 / 5 + 4 * c * c * si ** 2 * sj ** 2 / 9
            + 2 * si ** 2 * sj ** 2 / 9 - c * si ** 3 * sj / 2 - c * si * sj ** 3 / 2)
    np.testing.assert_allclose(R4, ref4, rtol=1e-11)


def test_pair_integral_matches_2d_adaptive_for_smooth_kernel():
    """Off-diagonal geometry (angle, node mapping) against scipy dblquad."""
    ell = 50.0
    g = lambda r: np.exp(-0.5 * (r / ell) ** 2)  # noqa: E731
    si, sj, th = 60.0, 80.0, 0.3
    ct = math.cos(th)
    ref = integrate.dblquad(
        lambda tp, t: math.exp(-0.5 * (t * t + tp * tp - 2 * t * tp * ct) / ell ** 2),
        0, si, 0, sj, epsabs=0, epsrel=1e-12)[0] / (si * sj)
    got = O.pair_R(np.array([si]), np.array([sj]), np.array([2 - 2 * ct]), g, 32)[0]
    assert got == pytest.approx(ref, rel=1e-11)


def test_diagonal_converges_to_1d_reduction():
    """R_ii -> (2/s^2) int_0^s (s - r) g(r) dr as Q grows (the kernel has a
    cusp at r = 0, so convergence is algebraic; the error is reported)."""
    L0, s = 20.0, 40.0
    g = lambda r: O.g_of_r(r, 1.0, L0)  # noqa: E731
    ex = 2 / s ** 2 * integrate.quad(lambda r: (s - r) * g(r), 0, s, epsabs=0,
                                     epsrel=1e-13, limit=500,
                                     points=[1e-6, 1e-3, 1e-1])[0]
    errs = [abs(O.pair_R(np.array([s]), np.array([s]), np.zeros(1), g, Q)[0] / ex - 1)
            for Q in (32, 64, 128, 256)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[1] < 5e-3 and errs[-1] < 5e-4


def test_constant_kernel_gives_constant_R():
    si, sj = np.array([123.0, 2000.0]), np.array([77.0, 2500.0])
    R = O.pair_R(si, sj, 2 - 2 * np.cos([0.1, 0.01]), lambda r: np.full_like(r, 0.7), 16)
    np.testing.assert_allclose(R, 0.7, rtol=1e-14)


# --------------------------------------------------------------- sparse K
@pytest.fixture(scope="module")
def small_cat():
    cat = make_catalogue("c1_plain_400", truth="mean")
    return catalogue_subset(cat, np.arange(150))


def test_neighbour_pairs_brute_force(small_cat):
    u = O.unit_vectors(small_cat["l"], small_cat["b"])
    x = u * small_cat["s"][:, None]
    c = small_cat["cutoff_pc"]
    pairs = O.neighbour_pairs(x, c)
    d2 = ((x[:, None] - x[None]) ** 2).sum(-1)
    i, j = np.nonzero(np.triu(d2 <= c * c, 1))
    np.testing.assert_array_equal(pairs, np.stack([i, j], 1))


def test_tapered_K_symmetric_positive_definite(small_cat):
    cv = O.build_cov(small_cat)
    K = cv["K"]
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0
    # sparse assembly agrees with dense
    cs = O.build_cov(small_cat, dense=False)
    np.testing.assert_array_equal(cs["K"].toarray(), K)


def test_small_variance_limit_lognormal_vs_linear(small_cat):
    """K_lognormal - K_linear = O(sigma2^2)."""
    diffs = []
    for s2 in (1e-2, 1e-3):
        c = dict(small_cat, sigma2=s2)
        Kl = O.build_cov(c, form=O.FORM_LOGNORMAL, Q=16)["K"]
        Kn = O.build_cov(c, form=O.FORM_LINEAR, Q=16)["K"]
        diffs.append(np.abs(Kl - Kn).max())
    assert 80 < diffs[0] / diffs[1] < 120


# -------------------------------------------------------------------- EP
def test_ep_with_gaussian_sites_is_gp_regression(small_cat):
    """Gaussian likelihood in ln A: one EP sweep gives exactly the noisy-GP
    conditional (Sect. 2 eq. cond_GP0), computed here by a plain solve."""
    cv = O.build_cov(small_cat)
    K, m = cv["K"], cv["m"]
    y = np.log(np.clip(small_cat["A_obs"], 1e-3, None))
    sa = small_cat["A_sigma"] / np.clip(small_cat["A_obs"], 1e-3, None)
    mean, var = O.gp_regression(K, m, y, sa ** 2)
    r = O.ep_run(K, m, y, sa, lik=O.LIK_GAUSS_IN_LNA, max_sweeps=3, tol=0.0)
    np.testing.assert_allclose(r["mu"], mean, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r["var"], var, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(r["tau"], 1 / sa ** 2, rtol=1e-9)


@pytest.mark.parametrize("case", [
    (math.log(3.0), 0.02, 3.1, 0.05),    # far star: sharp likelihood
    (math.log(0.1), 0.3, 0.1, 0.05),     # near star: likelihood plateau
    (math.log(0.3), 0.1, 0.25, 0.05),
    (math.log(0.2), 0.2, -0.05, 0.05),   # non-positive observation
    (0.0, 0.05, 1.0, 0.1),
])
def test_tilted_moments_rule_vs_adaptive(case):
    mc, vc, obs, sig = case
    m1, v1, _ = O.tilted_moments_gauss_in_a(mc, vc, obs, sig * sig)
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            m2, v2 = O.tilted_moments_adaptive(mc, vc, obs, sig * sig)
    assert m1 == pytest.approx(m2, abs=1e-10)
    assert v1 == pytest.approx(v2, rel=1e-9)


def test_tilted_log_normaliser_vs_adaptive():
    mc, vc, obs, s2 = math.log(0.5), 0.1, 0.45, 0.0025
    _, _, logZ = O.tilted_moments_gauss_in_a(mc, vc, obs, s2)
    f = lambda a: math.exp(-0.5 * (a - mc) ** 2 / vc - 0.5 * (obs - math.exp(a)) ** 2 / s2) \
        / math.sqrt(2 * math.pi * vc) / math.sqrt(2 * math.pi * s2)  # noqa: E731
    Z = integrate.quad(f, mc - 5, mc + 5, points=[math.log(obs)], epsabs=0,
                       epsrel=1e-12, limit=500)[0]
    assert logZ == pytest.approx(math.log(Z), abs=1e-10)


def test_single_star_ep_is_exact_posterior():
    """N = 1: the cavity is the prior, so converged EP reproduces the exact
    posterior moments, computed here by brute-force adaptive quadrature."""
    K = np.array([[0.15]])
    m = np.array([math.log(0.8)])
    obs, sig = np.array([0.65]), np.array([0.05])
    r = O.ep_run(K, m, obs, sig, max_sweeps=5, tol=1e-14)
    post = lambda a, k: a ** k * math.exp(-0.5 * (a - m[0]) ** 2 / K[0, 0]  # noqa: E731
                                          - 0.5 * (obs[0] - math.exp(a)) ** 2 / sig[0] ** 2)
    Z = [integrate.quad(post, -4, 3, args=(k,), epsabs=0, epsrel=1e-13,
                        limit=500, points=[math.log(0.65)])[0] for k in range(3)]
    mean = Z[1] / Z[0]
    var = Z[2] / Z[0] - mean ** 2
    assert r["mu"][0] == pytest.approx(mean, abs=1e-10)
    assert r["var"][0] == pytest.approx(var, rel=1e-8)


def test_ep_fixed_point_matches_tilted_moments(small_cat):
    """At convergence each site's tilted moments equal the posterior
    marginal (the moment-matching condition of eq. KL1')."""
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(80))
    cv = O.build_cov(cat)
    r = O.ep_run(cv["K"], cv["m"], cat["A_obs"], cat["A_sigma"], max_sweeps=60,
                 tol=1e-12)
    assert r["max_delta"] < 1e-12
    for i in range(0, 80, 7):
        tc = 1 / r["var"][i] - r["tau"][i]
        nc = r["mu"][i] / r["var"][i] - r["nu"][i]
        mh, vh, _ = O.tilted_moments_gauss_in_a(nc / tc, 1 / tc, cat["A_obs"][i],
                                                cat["A_sigma"][i] ** 2)
        assert mh == pytest.approx(r["mu"][i], abs=1e-9)
        assert vh == pytest.approx(r["var"][i], rel=1e-8)


def test_posterior_allows_zero_sites(small_cat):
    cv = O.build_cov(small_cat)
    n = len(cv["m"])
    mu, var, alpha = O.posterior(cv["K"], cv["m"], np.zeros(n), np.zeros(n))
    np.testing.assert_array_equal(mu, cv["m"])
    np.testing.assert_allclose(var, np.diag(cv["K"]), rtol=0, atol=0)


# -------------------------------------------------------------- predict
def test_predict_at_stars_equals_posterior(small_cat):
    cv = O.build_cov(small_cat)
    r = O.ep_run(cv["K"], cv["m"], small_cat["A_obs"], small_cat["A_sigma"],
                 max_sweeps=4, tol=0.0)
    idx = np.arange(0, 150, 13)
    mq, vq = O.predict(small_cat, cv["K"], cv["m"], r["tau"], r["nu"],
                       small_cat["l"][idx], small_cat["b"][idx], small_cat["s"][idx])
    np.testing.assert_allclose(mq, r["mu"][idx], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(vq, r["var"][idx], rtol=1e-9)


def test_predict_is_joint_gp_conditional(small_cat):
    """With Gaussian sites, prediction equals eq. cond_GP0 applied to the
    joint (stars + queries) covariance built by the same assembly."""
    rng = np.random.default_rng(5)
    nq = 12
    q = dict(l=rng.uniform(0, 1, nq) * math.pi / 180, b=rng.uniform(0, 1, nq) * math.pi / 180,
             s=np.exp(rng.uniform(math.log(100), math.log(3000), nq)))
    joint = dict(small_cat)
    for k in ("l", "b", "s"):
        joint[k] = np.concatenate([small_cat[k], q[k]])
    cvj = O.build_cov(joint)
    n = len(small_cat["s"])
    K, m = cvj["K"][:n, :n], cvj["m"][:n]
    y = np.log(np.clip(small_cat["A_obs"], 1e-3, None))
    sa = small_cat["A_sigma"] / np.clip(small_cat["A_obs"], 1e-3, None)
    Ks, Kss = cvj["K"][n:, :n], cvj["K"][n:, n:]
    C = K + np.diag(sa ** 2)
    mean_ref = cvj["m"][n:] + Ks @ linalg.solve(C, y - m, assume_a="pos")
    var_ref = np.diag(Kss - Ks @ linalg.solve(C, Ks.T, assume_a="pos"))
    tau, nu = 1 / sa ** 2, y / sa ** 2
    mq, vq = O.predict(small_cat, K, m, tau, nu, q["l"], q["b"], q["s"])
    np.testing.assert_allclose(mq, mean_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(vq, var_ref, rtol=1e-9, atol=1e-13)


def test_ep_two_stars_against_exact_posterior():
    """Multi-star EP has no closed form; for two correlated stars with the
    non-Gaussian likelihood A_obs ~ N(exp(a), sigma^2) the converged parallel
    EP posterior is compared with the exact posterior by integration on a
    grid (1601 x 1601 over +-8 prior sd): means within 1 % of the posterior
    sd, variances within 2 % (measured: 0.1 % and 0.7 %)."""
    m = np.array([-1.0, -0.7])
    K = np.array([[0.30, 0.18], [0.18, 0.25]])
    obs = np.array([0.45, 0.40])
    sig = np.array([0.15, 0.12])
    r = O.ep_run(K, m, obs, sig, max_sweeps=100, tol=1e-12)
    sd = np.sqrt(np.diag(K))
    g1 = np.linspace(m[0] - 8 * sd[0], m[0] + 8 * sd[0], 1601)
    g2 = np.linspace(m[1] - 8 * sd[1], m[1] + 8 * sd[1], 1601)
    A1, A2 = np.meshgrid(g1, g2, indexing="ij")
    Ki = np.linalg.inv(K)
    d1, d2 = A1 - m[0], A2 - m[1]
    logp = -0.5 * (Ki[0, 0] * d1 * d1 + 2 * Ki[0, 1] * d1 * d2 + Ki[1, 1] * d2 * d2)
    logp -= 0.5 * ((obs[0] - np.exp(A1)) / sig[0]) ** 2 + 0.5 * ((obs[1] - np.exp(A2)) / sig[1]) ** 2
    p = np.exp(logp - logp.max())
    Z = p.sum()
    mu = np.array([(p * A1).sum(), (p * A2).sum()]) / Z
    var = np.array([(p * (A1 - mu[0]) ** 2).sum(), (p * (A2 - mu[1]) ** 2).sum()]) / Z
    assert r["max_delta"] < 1e-12
    assert np.all(np.abs(r["mu"] - mu) < 0.01 * np.sqrt(var))
    assert np.all(np.abs(r["var"] / var - 1) < 0.02)


def test_sampled_posterior_equals_dense_posterior(small_cat):
    """The sparse-solve posterior (for catalogues whose dense K does not fit)
    reproduces the dense-Cholesky posterior."""
    cs = O.build_cov(small_cat, dense=False)
    cd = O.build_cov(small_cat)
    r = O.ep_run(cd["K"], cd["m"], small_cat["A_obs"], small_cat["A_sigma"], max_sweeps=3,
                 tol=0.0)
    idx = np.array([0, 5, 77, 149])
    mu, var = O.posterior_sampled(cs["K"], cs["m"], r["tau"], r["nu"], idx)
    mu0, v0, _ = O.posterior(cd["K"], cd["m"], r["tau"], r["nu"])
    np.testing.assert_allclose(mu, mu0, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(var, v0[idx], rtol=1e-9)


# ------------------------------------------------- prior moments of ln A
def _normal_expect(fn, m, v):
    """E[fn(a)] for a ~ N(m, v) by adaptive quadrature of the density."""
    sd = math.sqrt(v)
    val, _ = integrate.quad(lambda z: fn(m + sd * z) * math.exp(-0.5 * z * z),
                            -40.0, 40.0, epsabs=0, epsrel=1e-13, limit=400)
    return val / math.sqrt(2.0 * math.pi)


@pytest.mark.parametrize("s", [40.0, 300.0, 3000.0])
def test_prior_mean_and_variance_reproduce_extinction_moments(s):
    """Sect. 3 model: rho = e^f with E rho = rho_bar, so A = int_0^s rho dt has
    E[A] = rho_bar s and Var[A] = rho_bar^2 I_ss (I the double sightline
    integral of expm1(sigma2 phi)).  The lognormal form's prior N(m, K_ss) of
    a = ln A must reproduce both moments of A = e^a; the expectations are taken
    by integrating the normal density, not from the lognormal formulae."""
    rho_bar, sigma2, L0 = 1e-3, 1.0, 20.0
    cat = dict(l=np.array([0.3]), b=np.array([0.01]), s=np.array([s]), sigma2=sigma2,
               outer_scale_pc=L0, rho_bar=rho_bar, cutoff_pc=3 * L0, n_nodes=64)
    cv = O.build_cov(cat)
    m, Kss = float(cv["m"][0]), float(cv["diag"][0])
    R = float(O.pair_R([s], [s], [0.0], lambda r: O.g_of_r(r, sigma2, L0), 64)[0])
    EA = _normal_expect(math.exp, m, Kss)
    EA2 = _normal_expect(lambda a: math.exp(2 * a), m, Kss)
    assert EA == pytest.approx(rho_bar * s, rel=1e-10)
    assert EA2 - EA * EA == pytest.approx((rho_bar * s) ** 2 * R, rel=1e-9)
    assert Kss > 0.01   # large enough that a slip of K/2 in m would show


def test_linear_form_prior_mean_is_mean_log_density():
    """First-order form: a ~ ln s + (1/s) int f dt, so E[a] = ln s + E[f], with
    E[f] fixed by E[e^f] = rho_bar for f ~ N(E f, sigma2) (root-found here)."""
    from scipy import optimize
    rho_bar, sigma2 = 1e-3, 0.7
    mu_f = optimize.brentq(lambda mu: _normal_expect(math.exp, mu, sigma2) - rho_bar, -20, 0,
                           xtol=1e-14)
    s = np.array([100.0, 900.0])
    cat = dict(l=np.array([0.3, 0.3001]), b=np.array([0.01, 0.02]), s=s, sigma2=sigma2,
               outer_scale_pc=20.0, rho_bar=rho_bar, cutoff_pc=60.0, n_nodes=16)
    m = O.build_cov(cat, form=O.FORM_LINEAR)["m"]
    np.testing.assert_allclose(m, np.log(s) + mu_f, rtol=0, atol=1e-10)


# ----------------------------------------------------------- the taper
def test_wendland_values_at_tabulated_points():
    """Wendland (1995) psi_{3,1}(h) = (1-h)_+^4 (4h+1); values worked by hand."""
    h = np.array([0.0, 0.25, 0.5, 0.75, 0.9, 1.0, 1.5])
    want = np.array([1.0, 0.6328125, 0.1875, 0.015625, 0.00046, 0.0, 0.0])
    np.testing.assert_allclose(O.wendland(h), want, rtol=1e-14, atol=0)


def test_wendland_polynomial_structure():
    """psi_{3,1} is one quintic on [0, 1]: 1 - 10h^2 + 20h^3 - 15h^4 + 4h^5.
    No linear term and a cubic one: as a radial function of R^3 it is C^2 but
    not C^3 at the origin; at h = 1 it vanishes to fourth order.  The
    coefficients are recovered by a least-squares fit on [0, 1]."""
    h = np.linspace(0.0, 1.0, 41)
    coef = np.polynomial.polynomial.polyfit(h, O.wendland(h), 7)
    np.testing.assert_allclose(coef, [1, 0, -10, 20, -15, 4, 0, 0], rtol=0, atol=1e-8)
    assert np.all(O.wendland(np.array([1.0, 1.0 + 1e-12, 2.0, 10.0])) == 0.0)


def _radial_ft3(f, k):
    """Isotropic 3-D Fourier transform of a radial function supported in
    [0, 1]: (4 pi / k) int_0^1 r f(r) sin(k r) dr."""
    v, _ = integrate.quad(lambda r: r * f(r), 0.0, 1.0, weight="sin", wvar=k, limit=200)
    return 4.0 * math.pi / k * v


def test_wendland_is_positive_definite_in_3d():
    """The taper must be positive definite in R^3 (so K o W stays PD): its 3-D
    Fourier transform is non-negative.  The same check rejects the R^1 member
    psi_{2,1} = (1-h)^3 (3h+1), whose transform goes negative."""
    ks = np.linspace(0.1, 120.0, 1200)
    F = np.array([_radial_ft3(lambda r: float(O.wendland(np.array([r]))[0]), k) for k in ks])
    assert F.min() > -1e-12
    F21 = np.array([_radial_ft3(lambda r: (1 - r) ** 3 * (3 * r + 1), k) for k in ks])
    assert F21.min() < -1e-4
