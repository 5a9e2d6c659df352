"""Sampled posterior marginals of the 20,000-star bench workload against the
oracle's sparse-solve posterior with the same sites and the stored
covariance values: the FP32 form with exact variances, and the form the
bench times (tensor-core panel product, variances probed at twice the
cutoff, 64-vector deflated preconditioner)."""
import numpy as np
import pytest
from scipy import sparse

import oracle as O
from synth import make_catalogue

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as pkg
    return pkg


@pytest.mark.parametrize("form", ["exact", "bench"])
def test_bench_workload_sampled_marginals(gm, form):
    cat = make_catalogue("c2_plain_20k", truth="mean")
    n = len(cat["s"])
    extra = dict(probe_factor=2.0, deflate=64) if form == "bench" else {}
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, cg_tol=1e-6, **extra)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(2, 0.0)
        mu, var = ctx.get_posterior()
        tau, nu = ctx.get_sites()
        m0, _ = ctx.get_prior()
        perm = ctx.get_perm()
        rp, col, val = ctx.get_csr()
    # the stored K in the caller's order
    Kint = sparse.csr_matrix((val, col, rp), shape=(n, n))
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    K = Kint[inv][:, inv].tocsr()
    idx = np.random.default_rng(3).choice(n, 6, replace=False)
    mu_o, var_o = O.posterior_sampled(K, m0, tau, nu, idx, tol=1e-10)
    np.testing.assert_allclose(mu, mu_o, atol=1e-3)
    np.testing.assert_allclose(var[idx], var_o, rtol=1e-2)
