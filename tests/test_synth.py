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
