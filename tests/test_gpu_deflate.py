"""Spectral deflation of the FP32 preconditioner (variance panels and the
posterior-mean CG): the same posterior as plain Jacobi-PCG (within the FP32
panel tolerance) in fewer CG iterations, exact and probed."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("probe", [0.0, 2.0])
def test_deflated_panels_match_plain_in_fewer_iterations(gm, probe):
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(6000))
    out = {}
    for k in (0, 64):
        cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, cg_tol=1e-6,
                                       probe_factor=probe, deflate=k)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.build_cov()
            ctx.ep_sweep(2, 0.0)
            tau, nu = ctx.get_sites()
            mu, var = ctx.get_posterior()
            out[k] = (tau, nu, mu, var, ctx.stats())
    t0, n0, m0, v0, s0 = out[0]
    t1, n1, m1, v1, s1 = out[64]
    rel = np.abs(v1 - v0) / v0
    print("deflation (probe %g): variance CG iterations %d -> %d, mean CG %d -> %d; "
          "var rel max %.2e, mean %.2e" % (probe, s0["cg_iters_var"], s1["cg_iters_var"],
                                           s0["cg_iters_mean"], s1["cg_iters_mean"], rel.max(),
                                           np.abs(m1 - m0).max()))
    # both are FP32 panel solves stopped at 1e-5 relative residual
    assert rel.max() < 1e-3 and np.median(rel) < 1e-5
    assert np.abs(m1 - m0).max() < 1e-4
    assert s1["cg_iters_var"] < 0.7 * s0["cg_iters_var"]
    assert s1["cg_iters_mean"] < 0.8 * s0["cg_iters_mean"]
    # the refined mean solve reaches the same FP64-level residual
    assert s1["cg_resid_mean"] < 1e-5


@pytest.mark.parametrize("n,panel,probe", [(6000, 0, 2.0), (6000, 0, 0.0), (1337, 160, 2.0)])
def test_tensor_core_deflation_matches_cuda_core_form(gm, monkeypatch, n, panel, probe):
    """The tensor-core form of the deflated panel step (CG update fused with
    Y^T R, Yw C on tcgen05, BF16 planes written for the tile product) against
    the CUDA-core kernels: the same posterior within the FP32 panel tolerance
    and about the same iteration counts.  The second case has a ragged last
    column group (160 = 128 + 32), several panels and rows that fill neither
    a 16-row K-step nor a 128-row block."""
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(n))
    out = {}
    for form in ("0", "1"):
        monkeypatch.setenv("GM_DEFLATE_TC", form)
        cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP32, cg_tol=1e-6,
                                       probe_factor=probe, deflate=64, rhs_panel=panel)
        with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
            ctx.profile(True)
            ctx.build_cov()
            ctx.ep_sweep(2, 0.0)
            mu, var = ctx.get_posterior()
            out[form] = (mu, var, ctx.stats(), ctx.kernel_times())
            ctx.profile(False)
    m0, v0, s0, k0 = out["0"]
    m1, v1, s1, k1 = out["1"]
    assert "k_dtc_step" in k1 and "k_dtc_update" in k1
    assert "k_dtc_step" not in k0 and "k_df_update" in k0
    rel = np.abs(v1 - v0) / v0
    print("tensor-core deflation (n %d, panel %d, probe %g): variance CG iterations %d vs %d; "
          "var rel max %.2e median %.2e; mean max diff %.2e" % (n, panel, probe, s1["cg_iters_var"],
                                                   s0["cg_iters_var"], rel.max(), np.median(rel),
                                                   np.abs(m1 - m0).max()))
    assert rel.max() < 1e-3 and np.median(rel) < 1e-5
    assert np.abs(m1 - m0).max() < 1e-4
    # the panel loop looks at its active columns every 8 iterations, so the
    # counts move in steps of 8 when rounding moves one column across a check
    assert abs(s1["cg_iters_var"] - s0["cg_iters_var"]) <= 0.1 * s0["cg_iters_var"] + 8
