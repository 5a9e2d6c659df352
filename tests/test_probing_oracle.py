"""Pins of the probing statement (oracle/probing.py): the greedy colouring
against its definition by brute force, the exact special case against the
textbook posterior covariance (K^-1 + S)^-1, and the decay of the probing
error with the colour distance on a field of the 400-star workload.  (How
fast the error decays depends on the field: on this narrow 1-degree field
it is 4e-4 at twice the cutoff and 5e-6 at three times; on the 20,000-star
5-degree field it is 4e-8 at twice the cutoff.)"""
import numpy as np
import pytest

import oracle as O
from oracle import probing as P
from synth import catalogue_subset, make_catalogue


@pytest.fixture(scope="module")
def field():
    cat = make_catalogue("c1_plain_400", truth="mean")
    cat = catalogue_subset(cat, np.arange(260))
    cv = O.build_cov(cat)
    # site precisions of the size EP reaches: tau = (A / sigma_A)^2 in ln A;
    # a few very precise stars put the unit form to use
    A = np.clip(cat["A_obs"], 0.02, None)
    tau = (A / cat["A_sigma"]) ** 2
    tau[::17] *= 400.0
    return cat, cv, tau


def test_greedy_colouring_brute_force():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 10, size=(300, 3))
    D = 2.0
    col = P.greedy_colouring(x, D)
    d = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1))
    for i in range(len(x)):
        earlier = [col[j] for j in range(i) if d[i, j] < D]
        smallest = 0
        while smallest in earlier:
            smallest += 1
        assert col[i] == smallest
    same = (col[:, None] == col[None]) & ~np.eye(len(x), dtype=bool)
    assert d[same].min() >= D
    # greedy never needs more colours than the largest degree + 1
    assert col.max() + 1 <= ((d < D).sum(1)).max()


def test_all_distinct_colours_give_the_exact_posterior_variance(field):
    cat, cv, tau = field
    K = cv["K"]
    assert P.unit_form(K, tau).any() and not P.unit_form(K, tau).all()
    var = P.probed_variances(K, tau, np.arange(len(tau)))
    exact = np.diag(np.linalg.inv(np.linalg.inv(K) + np.diag(tau)))
    np.testing.assert_allclose(var, exact, rtol=1e-9)


def test_probing_error_decays_with_colour_distance(field):
    cat, cv, tau = field
    K = cv["K"]
    c = cat["cutoff_pc"]
    exact = np.diag(np.linalg.inv(np.linalg.inv(K) + np.diag(tau)))
    errs = {}
    for f in (0.25, 1.0, 3.0):
        col = P.greedy_colouring(cv["x"], f * c)
        assert col.max() + 1 < len(tau)          # the solves are actually shared
        var = P.probed_variances(K, tau, col)
        errs[f] = np.max(np.abs(var - exact) / exact)
    assert errs[0.25] > 1e-3                     # neighbours sharing a solve: wrong
    assert errs[3.0] < 3e-5
    assert errs[3.0] < errs[1.0] < errs[0.25]
