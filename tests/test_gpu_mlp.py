"""The tensor-core surrogate forward (tcgen05, two-piece BF16 operands, FP32
accumulation) against the FP64 statement of the network (oracle/mlp_oracle.py)
with the same FP32 weights, and the training kernels against its
backpropagation."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


def bf16(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def flat_params(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def forward_bf16(params, X):
    h = bf16(X)
    for k, (W, b) in enumerate(params):
        z = h @ bf16(W) + b.astype(np.float32)
        if k < len(params) - 1:
            h = bf16(M.silu(z))
        else:
            return z


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as pkg
    return pkg


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 40961])
def test_surrogate_forward_matches_cpu(gm, n):
    from synth import catalogue_subset, make_catalogue
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(4))
    rng = np.random.default_rng(n)
    params = M.init_params(7)
    # scale the last layer so both outputs are O(1) and sensitive to every unit
    params[-1] = (params[-1][0] * 0.5, np.array([0.3, -1.0]))
    si = np.exp(rng.uniform(np.log(100), np.log(3000), n))
    sj = si + rng.uniform(-60, 60, n)
    sj = np.clip(sj, 90, None)
    chord = rng.uniform(0, 0.02, n)
    sigma2, L0 = 1.0, 20.0
    cfg = gm.config_from_catalogue(cat)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        with pytest.raises(gm.GmError):
            ctx.surrogate_eval(si, sj, chord, sigma2, L0)   # no weights yet
        ctx.surrogate_set_params(flat_params(params))
        np.testing.assert_array_equal(ctx.surrogate_get_params(), flat_params(params))
        y, e = ctx.surrogate_eval(si, sj, chord, sigma2, L0)
    X = M.features(si, sj, chord, sigma2, L0)
    p32 = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
           for W, b in params]
    ref = M.forward(p32, X)[0]
    err_y = np.abs(y - ref[:, 0])
    err_e = np.abs(e - ref[:, 1])
    scale = 1 + np.abs(ref).max()
    # two-piece operands: each product to ~1e-5 relative, FP32 accumulation,
    # FP32 features and the fast exponential of SiLU
    assert np.median(err_y) < 1e-4 * scale and err_y.max() < 1e-3 * scale
    assert np.median(err_e) < 1e-4 * scale and err_e.max() < 1e-3 * scale
    # a single BF16 piece per operand would be ~1e-2: the split is what is measured
    if n >= 1000:
        one_piece = forward_bf16(params, X)
        assert np.median(np.abs(one_piece[:, 0] - ref[:, 0])) > 3 * np.median(err_y)


@pytest.mark.parametrize("kernel", ["tc", "simt"])
def test_surrogate_gradients_match_oracle(gm, monkeypatch, kernel):
    """The training gradients -- tensor-core forward/backward/weight-gradient
    kernel (two-piece BF16 operands, FP32 accumulation) or the FP32 CUDA-core
    kernels -- against the FP64 backpropagation of the oracle."""
    monkeypatch.setenv("GM_MLP_TRAIN", kernel)
    from synth import catalogue_subset, make_catalogue
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(4))
    rng = np.random.default_rng(11)
    params = M.init_params(3)
    n = 700
    X = rng.standard_normal((n, 5)).astype(np.float32)
    Y = rng.standard_normal(n).astype(np.float32)
    cfg = gm.config_from_catalogue(cat)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.surrogate_set_params(flat_params(params))
        loss, g = ctx.surrogate_grad(X, Y, 0.1)
    p32 = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
           for W, b in params]
    lo, go = M.loss_and_grads(p32, X.astype(np.float64), Y.astype(np.float64), lam=0.1)
    assert loss == pytest.approx(lo, rel=1e-4)
    gref = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in go])
    np.testing.assert_allclose(g, gref, rtol=2e-3, atol=2e-5 * np.abs(gref).max())


def test_surrogate_training_assembly_and_posterior(gm):
    """Train on the GPU, assemble K with the surrogate (quadrature fallback at
    the gate), and measure the entries' error and the posterior error it
    induces against the quadrature path."""
    from synth import make_catalogue
    cat = make_catalogue("c1_plain_400")
    base = dict(precision=gm.PREC_FP32, cg_tol=1e-7)
    with gm.ep_init(gm.config_from_catalogue(cat, **base), cat["l"], cat["b"], cat["s"],
                    cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        rp, col, Kq = ctx.get_csr()
        ctx.ep_sweep(5)
        mu_q, var_q = ctx.get_posterior()
    cfg = gm.config_from_catalogue(cat, cov_source=gm.COV_SURROGATE, **base)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        st = ctx.surrogate_train(n_pairs=500_000, steps=6000, batch=4096, lr=3e-3, seed=5)
        assert st["surrogate_val_rmse"] < 0.06, st
        ctx.build_cov()
        rp2, col2, Ks = ctx.get_csr()
        st = ctx.stats()
        ctx.ep_sweep(5)
        mu_s, var_s = ctx.get_posterior()
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    # the gate bounds the estimated error of each served (tapered) entry at
    # 1e-4; the error head tracks the 95th percentile, so a few served entries
    # exceed it, by a small factor
    err = np.abs(Ks - Kq)
    served_mask = err > 0
    assert err.max() < 5e-4, err.max()
    served = st["n_pairs"] - 400 - st["surrogate_fallback"]
    assert served > 0.15 * (st["n_pairs"] - 400), st
    # posterior error induced by the surrogate, against the quadrature path:
    # within the 1e-3 equal-error bar on the mean of ln A
    mu_err = np.abs(mu_s - mu_q).max()
    var_err = np.max(np.abs(var_s - var_q) / var_q)
    print("surrogate posterior error: mean ln A %.2e, var rel %.2e, served %d of %d pairs "
          "(%d entries changed)" % (mu_err, var_err, served, st["n_pairs"] - 400,
                                    int(served_mask.sum())))
    assert mu_err < 1e-3
    assert var_err < 2e-3
