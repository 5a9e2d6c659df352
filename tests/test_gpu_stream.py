"""Streamed assembly of covariance row blocks (gm_cov_rows) against the
stored covariance of gm_build_cov and the oracle's pair integral."""
import numpy as np
import pytest

import oracle as O
from synth import catalogue_subset, make_catalogue

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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_row_blocks_equal_the_stored_rows(gm, prec):
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(3000))
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    cfg = gm.config_from_catalogue(cat, precision=p)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        blocks = [ctx.cov_rows(r0, nr) for r0, nr in ((0, 700), (700, 1), (701, 2299))]
        ctx.build_cov()
        rp, col, val = ctx.get_csr()
    rp_b = np.concatenate([blocks[0][0]] + [b[0][1:] + off for b, off in
                                           zip(blocks[1:], np.cumsum([b[0][-1] for b in blocks])[:-1])])
    col_b = np.concatenate([b[1] for b in blocks])
    val_b = np.concatenate([b[2] for b in blocks]).astype(np.float64)
    np.testing.assert_array_equal(rp_b, rp)
    np.testing.assert_array_equal(col_b, col)
    # the stored lower triangle mirrors the upper entries, the blocks compute
    # every entry from its own row: equal up to the summation order
    np.testing.assert_allclose(val_b, val, rtol=1e-11 if prec == "fp64" else 5e-6, atol=0)
    assert all(b[3] == 0 for b in blocks)


def test_surrogate_row_block_against_quadrature_and_oracle(gm):
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(3000))
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, cov_source=gm.COV_SURROGATE,
                                   quad_rule=gm.QUAD_BAND)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.surrogate_train(n_pairs=500_000, steps=3000, batch=8192, lr=3e-3)
        rp, col, val_s, fb = ctx.cov_rows(0, 600)
        _, col_q, val_q, fq = ctx.cov_rows(0, 600, source=gm.COV_QUADRATURE)
        perm = ctx.get_perm()
    np.testing.assert_array_equal(col, col_q)
    assert fq == 0 and 600 <= fb < len(col)          # the diagonal always falls back
    d = np.abs(val_s.astype(np.float64) - val_q)
    # entries the network served are within a few times the gate of the rule
    assert np.mean(d > 10 * cfg.surrogate_gate) < 0.01, np.mean(d > 10 * cfg.surrogate_gate)
    # the block's quadrature entries against the oracle's band rule on a sample
    from oracle import band as Bd
    rows = np.repeat(np.arange(600), np.diff(rp))
    rng = np.random.default_rng(0)
    k = rng.choice(len(col), 60, replace=False)
    i, j = perm[rows[k]], perm[col[k]]
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * cat["s"][:, None]
    g = lambda r: O.g_of_r(r, float(cat["sigma2"]), float(cat["outer_scale_pc"]))
    R = Bd.pair_R_band(cat["s"][i], cat["s"][j], ((u[i] - u[j]) ** 2).sum(1), g,
                       float(cat["outer_scale_pc"]), n=6, h0=1e-3, q=3.0, m0=0.25, K=40.0)[0]
    K = np.log1p(R) * O.wendland(np.linalg.norm(x[i] - x[j], axis=1) / float(cat["cutoff_pc"]))
    np.testing.assert_allclose(val_q[k], K, rtol=2e-5, atol=1e-9)
