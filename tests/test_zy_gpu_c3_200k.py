"""The 200,000-star workload (10 x 10 deg, outer scale 10 pc, 64 nodes) at
full size: the covariance checked on sampled entries against the oracle's
pair integral and on the neighbour structure of sampled rows, the probing
colouring on sampled stars, and one EP sweep."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

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


def test_c3_full_size_sampled(gm):
    cat = make_catalogue("c3_mixed_200k")
    n = len(cat["s"])
    c = float(cat["cutoff_pc"])
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * cat["s"][:, None]
    tree = cKDTree(x)
    rng = np.random.default_rng(0)
    rows = rng.choice(n, 200, replace=False)
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, probe_factor=2.0)
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        st = ctx.stats()
        # sampled pairs: up to 8 neighbours of each sampled row (within the
        # cutoff by brute force) and up to 4 partners just beyond it
        I, J, inside = [], [], []
        for r, nb in zip(rows, tree.query_ball_point(x[rows], c)):
            nb = np.array(nb)
            k = min(8, len(nb))
            I += [r] * k
            J += list(rng.choice(nb, k, replace=False))
            inside += [True] * k
            far = np.array(tree.query_ball_point(x[r], 1.3 * c))
            d = np.linalg.norm(x[far] - x[r], axis=1)
            out = far[d > c][:4]
            I += [r] * len(out)
            J += list(out)
            inside += [False] * len(out)
        I, J, inside = np.array(I), np.array(J), np.array(inside)
        vals = ctx.get_entries(I, J)
        kd = ctx.get_prior()[1]
        col = ctx.get_probe_colours()
        ctx.ep_sweep(1)
        tau, nu = ctx.get_sites()
        st1 = ctx.stats()
    assert st["nnz"] > 5e8 and st["probe_colours"] < n
    # entries beyond the cutoff are not stored
    assert np.all(vals[~inside] == 0.0)
    # stored entries against the oracle's pair integral (same node rule, taper)
    g = lambda r: O.g_of_r(r, float(cat["sigma2"]), float(cat["outer_scale_pc"]))
    i, j = I[inside], J[inside]
    chord2 = ((u[i] - u[j]) ** 2).sum(1)
    K = O.K_from_R(O.pair_R(cat["s"][i], cat["s"][j], chord2, g, int(cat["n_nodes"])),
                   O.FORM_LOGNORMAL)
    d = np.linalg.norm(x[i] - x[j], axis=1)
    K = K * O.wendland(d / c)
    np.testing.assert_allclose(vals[inside], K, rtol=2e-5, atol=1e-7 * K.max())
    kd_ref = O.K_from_R(O.pair_R(cat["s"][rows], cat["s"][rows], np.zeros(len(rows)), g,
                                 int(cat["n_nodes"])), O.FORM_LOGNORMAL)
    np.testing.assert_allclose(kd[rows], kd_ref, rtol=2e-5)
    # colouring: sampled stars differ in colour from every star closer than 2c
    for r, nb in zip(rows, tree.query_ball_point(x[rows], np.nextafter(2 * c, 0.0))):
        others = [q for q in nb if q != r]
        assert col[r] not in set(col[others])
    # one sweep from zero sites: every site finite, few skipped
    assert np.all(np.isfinite(tau)) and np.all(np.isfinite(nu))
    assert st1["sites_skipped"] < 0.01 * n
    print("c3 full size: nnz %d, %d probing classes, %d skipped" %
          (st["nnz"], st["probe_colours"], st1["sites_skipped"]))
