"""Several independent fields solved together in one context (block-diagonal
K, packed multi-field variance panels, graph-captured CG) against the FP64
oracle per field and against one context per field."""
import numpy as np
import pytest

import oracle as O
from synth import make_fields

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


def concat(fields):
    keys = ("l", "b", "s", "A_obs", "A_sigma")
    cat = {k: np.concatenate([f[k] for f in fields]) for k in keys}
    fid = np.concatenate([np.full(len(f["s"]), i, dtype=np.int32) for i, f in enumerate(fields)])
    L0 = np.array([f["outer_scale_pc"] for f in fields])
    return cat, fid, L0


def test_fields_match_oracle_and_single_contexts(gm):
    fields = make_fields(n_fields=5, scale=0.06, seed=2)   # ~30-480 stars each
    cat, fid, L0 = concat(fields)
    # interleave the stars of different fields in caller order
    order = np.random.default_rng(0).permutation(len(fid))
    cat = {k: v[order] for k, v in cat.items()}
    fid = fid[order]
    base = dict(sigma2=1.0, outer_scale_pc=20.0, rho_bar=1e-3, cutoff_pc=60.0, n_nodes=32,
                quad_rule=gm.QUAD_GL, precision=gm.PREC_FP32, cg_tol=1e-7)
    cfg = gm.default_config(**base)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"],
                    field_id=fid, field_L0=L0, field_cutoff=3 * L0) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(4)
        mu, var = ctx.get_posterior()
        st = ctx.stats()
    assert st["sites_skipped"] >= 0
    for f, fc in enumerate(fields):
        sel = fid == f
        fcat = dict(fc, n_nodes=32, cutoff_pc=3 * fc["outer_scale_pc"])
        # one context per field
        cfg1 = gm.default_config(**dict(base, outer_scale_pc=fc["outer_scale_pc"],
                                        cutoff_pc=3 * fc["outer_scale_pc"]))
        with gm.ep_init(cfg1, fc["l"], fc["b"], fc["s"], fc["A_obs"], fc["A_sigma"]) as c1:
            c1.build_cov()
            c1.ep_sweep(4)
            m1, v1 = c1.get_posterior()
        # caller order inside the batch: stars of field f appear in the order of `order`
        idx = order[sel] - sum(len(g["s"]) for g in fields[:f])
        np.testing.assert_allclose(mu[sel], m1[idx], rtol=0, atol=2e-4)
        np.testing.assert_allclose(var[sel], v1[idx], rtol=5e-3)
        cv = O.build_cov(fcat)
        r = O.ep_run(cv["K"], cv["m"], fc["A_obs"], fc["A_sigma"], max_sweeps=4, tol=0.0)
        np.testing.assert_allclose(mu[sel], r["mu"][idx], rtol=0, atol=1e-3)
        np.testing.assert_allclose(var[sel], r["var"][idx], rtol=1e-2)
