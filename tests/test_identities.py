"""Identities the CUDA path relies on, checked on the oracle's dense
matrices (CPU): the site-form posterior and the unit-right-hand-side
variance formula used for site-dominated stars."""
import numpy as np
from scipy import linalg

import oracle as O
from synth import catalogue_subset, make_catalogue


def test_unit_rhs_variance_identity():
    """With B = I + S^1/2 K S^1/2: Sigma = (K^-1 + S)^-1 has
    Sigma_ii = K_ii - v_i^T B^-1 v_i (v_i = S^1/2 K e_i) = (1 - (B^-1)_ii) / tau_i,
    and the cavity precision 1/Sigma_ii - tau_i = tau_i y_i / (1 - y_i)."""
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(120))
    cv = O.build_cov(cat)
    K = cv["K"]
    rng = np.random.default_rng(3)
    tau = rng.uniform(0.5, 4000.0, 120)
    d = np.sqrt(tau)
    B = np.eye(120) + d[:, None] * K * d[None, :]
    Binv = linalg.inv(B)
    Sigma = linalg.inv(linalg.inv(K) + np.diag(tau))
    V = d[:, None] * K
    form_v = np.diag(K) - np.einsum("ij,ij->j", V, Binv @ V)
    y = np.diag(Binv)
    form_e = (1 - y) / tau
    np.testing.assert_allclose(form_v, np.diag(Sigma), rtol=1e-8)
    np.testing.assert_allclose(form_e, np.diag(Sigma), rtol=1e-8)
    np.testing.assert_allclose(1 / np.diag(Sigma) - tau, tau * y / (1 - y), rtol=1e-6)
