"""The synthetic-input generator: seeded, shaped like the workloads, and its
truth simulator has the mean the model fixes (E[A] = rho_bar * s)."""
import numpy as np

from synth import WORKLOADS, Workload, catalogue_subset, make_catalogue, make_fields


def test_seeded_and_in_field():
    a = make_catalogue("c1_plain_400", truth="mean")
    b = make_catalogue("c1_plain_400", truth="mean")
    for k in ("l", "b", "s", "A_obs"):
        np.testing.assert_array_equal(a[k], b[k])
    wl = WORKLOADS["c1_plain_400"]
    assert len(a["s"]) == wl.n
    assert a["s"].min() >= 100 and a["s"].max() <= 3000
    deg = 180 / np.pi
    assert (a["l"] * deg).min() >= 0 and (a["l"] * deg).max() <= 1
    assert (a["b"] * deg).min() >= 0 and (a["b"] * deg).max() <= 1


def test_truth_mean_extinction_is_rho_bar_s():
    """Monte Carlo over independent fields: A_true / (rho_bar s) averages to 1
    (the log-density mean is ln rho_bar - sigma2/2)."""
    ratios = []
    for seed in range(12):
        wl = Workload("t", 40, (0.0, 20.0), (0.0, 20.0), s_pc=(30.0, 60.0),
                      outer_scale_pc=4.0, seed=seed)
        c = make_catalogue(wl)
        ratios.append(np.mean(c["A_true"] / (wl.rho_bar * c["s"])))
    ratios = np.array(ratios)
    se = ratios.std(ddof=1) / np.sqrt(len(ratios))
    assert abs(ratios.mean() - 1.0) < 4 * se + 0.02


def test_fields_and_subset():
    f = make_fields(n_fields=4, scale=0.05, seed=3)
    assert len(f) == 4 and all(len(c["s"]) >= 1 for c in f)
    c = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(10))
    assert len(c["l"]) == 10 and c["sigma2"] == 1.0


def _truth_draws(order, n_draws=400):
    """Extinctions of 6 stars (60-140 pc, outer scale 20 pc) over independent
    draws of the spectrally synthesised field, and the model covariance
    rho_bar^2 I_ij of Sect. 3 (converged band rule of the oracle)."""
    import oracle as O
    from oracle import band as Bd
    from synth.catalogue import _field_positions, _truth_fft
    L0, sigma2, rho = 20.0, 1.0, 1e-3
    l, b, s = _field_positions(np.random.default_rng(5), 6, (0.0, 4.0), (0.0, 4.0),
                               (60.0, 140.0))
    A = np.array([_truth_fft(np.random.default_rng([7, k]), l, b, s, sigma2, L0, rho,
                             order=order) for k in range(n_draws)])
    u = O.unit_vectors(l, b)
    g = lambda r: O.g_of_r(r, sigma2, L0)  # noqa: E731
    n = len(s)
    M = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            R, _ = Bd.pair_R_band(s[i], s[j], ((u[i] - u[j]) ** 2).sum(), g, L0)
            M[i, j] = M[j, i] = rho * rho * R[0] * s[i] * s[j]
    return A, s, rho, M


def test_truth_covariance_matches_the_model():
    """Monte Carlo of the truth simulator (nearest-cell reading of the field):
    E[A] = rho_bar s and Cov(A_i, A_j) = rho_bar^2 I_ij, the lognormal moment
    match of Sect. 3 with g = expm1(sigma2 phi), within the sampling error of
    400 draws (about 3 % on the mean, 8 % on variances)."""
    A, s, rho, M = _truth_draws(order=0)
    C = np.cov(A.T)
    iu = np.triu_indices(len(s), 1)
    assert abs(np.mean(A.mean(0) / (rho * s)) - 1.0) < 0.05
    assert abs(np.mean(np.diag(C) / np.diag(M)) - 1.0) < 0.1
    assert abs(np.mean(C[iu] / M[iu]) - 1.0) < 0.1


def test_trilinear_reading_lowers_the_field_variance():
    """Trilinear interpolation of 2 pc cells averages values whose
    correlation is about 0.8 (the Kolmogorov cusp), so the sampled
    log-density has less variance and E[exp f] < rho_bar."""
    A, s, rho, M = _truth_draws(order=1)
    assert np.mean(A.mean(0) / (rho * s)) < 0.97
    assert np.mean(np.diag(np.cov(A.T)) / np.diag(M)) < 0.95
