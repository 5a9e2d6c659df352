"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, derived from the arithmetic:
  FP64 mode: covariance entries 1e-9 relative (cubic-table interpolation of
  the log-density kernel, < 2e-12 of g(0)); posterior means/variances 1e-6
  relative (the target the method is held to).
  FP32 mode: covariance entries 2e-5 relative (FP32 sums of Q^2 products);
  posterior mean ln A within 1e-3 absolute and variances within 1e-2
  relative (FP32 CG, FP64-refined mean).
Structure (CSR pattern, permutation) is compared exactly.
"""
import math

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


@pytest.fixture(scope="module")
def c1():
    return make_catalogue("c1_plain_400")


@pytest.fixture(scope="module")
def c1_oracle(c1):
    cv = O.build_cov(c1)
    return cv


def init(gm, cat, **kw):
    cfg = gm.config_from_catalogue(cat, **kw)
    return gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"])


def csr_external(ctx):
    """GPU CSR mapped to caller indices: dict of (i, j) -> value."""
    rp, col, val = ctx.get_csr()
    perm = ctx.get_perm()
    rows = np.repeat(np.arange(ctx.n), np.diff(rp))
    return perm[rows], perm[col], val


def dense_from_gpu(ctx):
    i, j, v = csr_external(ctx)
    K = np.zeros((ctx.n, ctx.n))
    K[i, j] = v
    return K


def oracle_pattern(n, pairs):
    P = np.zeros((n, n), dtype=bool)
    P[pairs[:, 0], pairs[:, 1]] = True
    P[pairs[:, 1], pairs[:, 0]] = True
    P[np.arange(n), np.arange(n)] = True
    return P


# ------------------------------------------------------------------ covariance
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_covariance_matches_oracle_c1(gm, c1, c1_oracle, prec):
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    with init(gm, c1, precision=p) as ctx:
        nnz = ctx.build_cov()
        i, j, v = csr_external(ctx)
        perm = ctx.get_perm()
        m, kd = ctx.get_prior()
        rp, col, _ = ctx.get_csr()
    n = len(c1["s"])
    assert sorted(perm.tolist()) == list(range(n))
    # rows sorted, pattern exact
    for r in range(n):
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)
    P = np.zeros((n, n), dtype=bool)
    P[i, j] = True
    np.testing.assert_array_equal(P, oracle_pattern(n, c1_oracle["pairs"]))
    assert nnz == n + 2 * len(c1_oracle["pairs"])
    Ko = c1_oracle["K"][i, j]
    rtol = 1e-9 if prec == "fp64" else 2e-5
    # FP32: the taper (1 - h)^4 (4h + 1) near the cutoff has relative error
    # ~4 eps_32 / (1 - h), so entries within 1 % of the cutoff (below 1e-6)
    # get an absolute floor of 1e-10
    np.testing.assert_allclose(v, Ko, rtol=rtol, atol=1e-12 if prec == "fp64" else 1e-10)
    np.testing.assert_allclose(kd, c1_oracle["diag"], rtol=rtol)
    np.testing.assert_allclose(m, c1_oracle["m"], rtol=rtol, atol=rtol)


def test_covariance_multi_tile_ragged(gm):
    """2,531 stars of the 5x5 deg field: many warps, cells and a ragged tail."""
    cat = catalogue_subset(make_catalogue("c2_plain_20k", truth="mean"), np.arange(2531))
    cat["n_nodes"] = 24
    with init(gm, cat, precision=gm.PREC_FP64) as ctx:
        ctx.build_cov()
        i, j, v = csr_external(ctx)
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * cat["s"][:, None]
    pairs = O.neighbour_pairs(x, cat["cutoff_pc"])
    got = set(zip(i.tolist(), j.tolist()))
    want = set(zip(pairs[:, 0].tolist(), pairs[:, 1].tolist()))
    want |= set((b, a) for a, b in want) | set((k, k) for k in range(2531))
    assert got == want
    # values on a sample of entries
    rng = np.random.default_rng(0)
    pick = rng.choice(len(i), 400, replace=False)
    ii, jj = i[pick], j[pick]
    chord2 = ((u[ii] - u[jj]) ** 2).sum(1)
    g = lambda r: O.g_of_r(r, 1.0, 20.0)  # noqa: E731
    R = O.pair_R(cat["s"][ii], cat["s"][jj], chord2, g, 24)
    d = np.sqrt(((x[ii] - x[jj]) ** 2).sum(1))
    ref = np.log1p(R) * O.wendland(d / cat["cutoff_pc"])
    np.testing.assert_allclose(v[pick], ref, rtol=1e-9, atol=1e-13)


# ------------------------------------------------------------------ EP
def test_gaussian_sites_reproduce_gp_regression(gm, c1, c1_oracle):
    """Likelihood Gaussian in ln A: one sweep = eq. cond_GP0 exactly."""
    y = np.log(np.clip(c1["A_obs"], 1e-3, None))
    sa = c1["A_sigma"] / np.clip(c1["A_obs"], 1e-3, None)
    cat = dict(c1, A_obs=y, A_sigma=sa)
    with init(gm, cat, precision=gm.PREC_FP64, likelihood=gm.LIK_GAUSS_IN_LNA) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(1)
        mu, var = ctx.get_posterior()
        tau, nu = ctx.get_sites()
    mean, v = O.gp_regression(c1_oracle["K"], c1_oracle["m"], y, sa ** 2)
    np.testing.assert_allclose(tau, 1 / sa ** 2, rtol=1e-9)
    np.testing.assert_allclose(mu, mean, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(var, v, rtol=1e-7)


@pytest.fixture(scope="module")
def c1_ep5(c1, c1_oracle):
    return O.ep_run(c1_oracle["K"], c1_oracle["m"], c1["A_obs"], c1["A_sigma"], max_sweeps=5,
                    tol=0.0)


def test_ep_fp64_matches_oracle(gm, c1, c1_ep5):
    with init(gm, c1, precision=gm.PREC_FP64) as ctx:
        ctx.build_cov()
        done, delta = ctx.ep_sweep(5, 0.0)
        mu, var = ctx.get_posterior()
        tau, nu = ctx.get_sites()
        st = ctx.stats()
    assert done == 5 and st["sites_skipped"] == 0
    np.testing.assert_allclose(tau, c1_ep5["tau"], rtol=1e-6)
    np.testing.assert_allclose(nu, c1_ep5["nu"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(mu, c1_ep5["mu"], rtol=1e-6)
    np.testing.assert_allclose(var, c1_ep5["var"], rtol=1e-6)


def test_ep_fp32_matches_oracle_within_form_tolerance(gm, c1, c1_ep5):
    with init(gm, c1, precision=gm.PREC_FP32, cg_tol=1e-7) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(5, 0.0)
        mu, var = ctx.get_posterior()
    np.testing.assert_allclose(mu, c1_ep5["mu"], rtol=0, atol=1e-3)
    np.testing.assert_allclose(var, c1_ep5["var"], rtol=1e-2)


def test_predict_matches_oracle(gm, c1, c1_oracle, c1_ep5):
    rng = np.random.default_rng(7)
    nq = 50
    lq = rng.uniform(0, 1, nq) * math.pi / 180
    bq = rng.uniform(0, 1, nq) * math.pi / 180
    sq = np.exp(rng.uniform(math.log(90), math.log(3100), nq))
    # include the first 5 stars themselves: prediction there is the posterior
    lq[:5], bq[:5], sq[:5] = c1["l"][:5], c1["b"][:5], c1["s"][:5]
    with init(gm, c1, precision=gm.PREC_FP64) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(5, 0.0)
        mq, vq = ctx.predict(lq, bq, sq)
    mo, vo = O.predict(c1, c1_oracle["K"], c1_oracle["m"], c1_ep5["tau"], c1_ep5["nu"], lq, bq, sq)
    np.testing.assert_allclose(mq, mo, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(vq, vo, rtol=1e-6, atol=1e-10)
    np.testing.assert_allclose(mq[:5], c1_ep5["mu"][:5], rtol=1e-6)


# ------------------------------------------------------------------ edges
def test_skip_rule_matches_oracle(gm):
    """The 600 nearest stars of the 5x5 deg field include weak positive
    observations whose tilted distribution is wider than the cavity (the
    likelihood is not log-concave there): both sides skip the same updates,
    sweep by sweep, and end with the same sites."""
    cat = make_catalogue("c2_plain_20k", truth="mean")
    sub = catalogue_subset(cat, np.sort(np.argsort(cat["s"])[:600]))
    sub = dict(sub, n_nodes=32)   # the rule under test does not depend on Q
    cv = O.build_cov(sub)
    tau, nu = np.zeros(600), np.zeros(600)
    with init(gm, sub, precision=gm.PREC_FP64) as ctx:
        ctx.build_cov()
        total = 0
        for sweep in range(3):
            tau, nu, _, sk, _, _ = O.ep_sweep(cv["K"], cv["m"], sub["A_obs"], sub["A_sigma"], tau, nu)
            ctx.ep_sweep(1)
            assert ctx.stats()["sites_skipped"] == sk, sweep
            total += sk
        tg, ng = ctx.get_sites()
    assert total > 0
    np.testing.assert_allclose(tg, tau, rtol=1e-6)
    np.testing.assert_allclose(ng, nu, rtol=1e-6, atol=1e-6)


def test_single_star(gm):
    cat = catalogue_subset(make_catalogue("c1_plain_400"), np.arange(1))
    with init(gm, cat, precision=gm.PREC_FP64) as ctx:
        assert ctx.build_cov() == 1
        ctx.ep_sweep(3)
        mu, var = ctx.get_posterior()
    cv = O.build_cov(cat)
    r = O.ep_run(cv["K"], cv["m"], cat["A_obs"], cat["A_sigma"], max_sweeps=3, tol=0.0)
    np.testing.assert_allclose(mu, r["mu"], rtol=1e-9)
    np.testing.assert_allclose(var, r["var"], rtol=1e-8)


def test_isolated_and_coincident_sightlines(gm):
    """Stars far apart (empty off-diagonal rows), two stars on one sightline
    (theta = 0) and two identical directions at equal distance (s_i = s_j)."""
    l = np.radians([0.0, 10.0, 20.0, 30.0, 30.0, 40.0, 40.0])
    b = np.radians([0.0, 0.0, 0.0, 1.0, 1.0, 2.0, 2.0])
    s = np.array([500.0, 800.0, 1200.0, 700.0, 730.0, 300.0, 300.0])
    obs = 1e-3 * s * np.array([1.1, 0.9, 1.0, 1.05, 1.0, 0.95, 1.02])
    sig = np.full(7, 0.05)
    cat = dict(l=l, b=b, s=s, A_obs=obs, A_sigma=sig, sigma2=1.0, outer_scale_pc=20.0,
               rho_bar=1e-3, cutoff_pc=60.0, n_nodes=32)
    with init(gm, cat, precision=gm.PREC_FP64) as ctx:
        nnz = ctx.build_cov()
        ctx.ep_sweep(4)
        mu, var = ctx.get_posterior()
        K = dense_from_gpu(ctx)
    cv = O.build_cov(cat)
    assert nnz == 7 + 4
    np.testing.assert_allclose(K, cv["K"], rtol=1e-9, atol=1e-14)
    r = O.ep_run(cv["K"], cv["m"], obs, sig, max_sweeps=4, tol=0.0)
    np.testing.assert_allclose(mu, r["mu"], rtol=1e-7)
    np.testing.assert_allclose(var, r["var"], rtol=1e-6)


def test_rerun_is_bit_identical_and_resume_matches(gm, c1):
    """Cold-started solves: reruns and save/restore are bit-identical."""
    def run(n):
        with init(gm, c1, precision=gm.PREC_FP64, warm_start=0) as ctx:
            ctx.build_cov()
            ctx.ep_sweep(n)
            return ctx.get_sites(), ctx.get_posterior()
    (t1, n1), (m1, v1) = run(4)
    (t2, n2), (m2, v2) = run(4)
    assert np.array_equal(t1, t2) and np.array_equal(m1, m2) and np.array_equal(v1, v2)
    (ta, na), _ = run(2)
    with init(gm, c1, precision=gm.PREC_FP64, warm_start=0) as ctx:
        ctx.build_cov()
        ctx.set_sites(ta, na)
        ctx.ep_sweep(2)
        (tb, nb) = ctx.get_sites()
        mb, vb = ctx.get_posterior()
    assert np.array_equal(tb, t1) and np.array_equal(nb, n1)
    assert np.array_equal(mb, m1) and np.array_equal(vb, v1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_warm_started_variances_agree_with_cold(gm, c1, prec):
    p = gm.PREC_FP64 if prec == "fp64" else gm.PREC_FP32
    out = []
    for warm in (0, 1):
        with init(gm, c1, precision=p, warm_start=warm) as ctx:
            ctx.build_cov()
            ctx.ep_sweep(4)
            out.append(ctx.get_posterior())
    rtol = 1e-8 if prec == "fp64" else 2e-3
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=rtol, atol=rtol)
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=rtol)


def test_call_order_and_bad_sites(gm, c1):
    with init(gm, c1) as ctx:
        with pytest.raises(gm.GmError) as e:
            ctx.ep_sweep(1)
        assert e.value.status == 8
        ctx.build_cov()
        bad = np.zeros(len(c1["s"]))
        bad[3] = -1.0
        with pytest.raises(gm.GmError) as e:
            ctx.set_sites(bad, np.zeros_like(bad))
        assert e.value.status == 1
    bad = dict(c1, s=np.where(np.arange(400) == 5, -1.0, c1["s"]))
    with pytest.raises(gm.GmError) as e:
        init(gm, bad)
    assert e.value.status == 1


def test_device_pointer_inputs_and_outputs(gm, c1):
    import torch
    dev = torch.device("cuda:0")
    T = {k: torch.tensor(c1[k], dtype=torch.float64, device=dev)
         for k in ("l", "b", "s", "A_obs", "A_sigma")}
    cfg = gm.config_from_catalogue(c1)
    with gm.ep_init(cfg, T["l"], T["b"], T["s"], T["A_obs"], T["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(2)
        out = (torch.empty(400, dtype=torch.float64, device=dev),
               torch.empty(400, dtype=torch.float64, device=dev))
        ctx.get_posterior(out=out)
        mh, vh = ctx.get_posterior()
    np.testing.assert_array_equal(out[0].cpu().numpy(), mh)
    np.testing.assert_array_equal(out[1].cpu().numpy(), vh)


# ------------------------------------------------------------------ full size
def test_bench_workload_full_size_fp32(gm):
    """20,000 stars (the benchmark workload), FP32 form as timed: exact CSR
    pattern against the oracle's neighbour search, sampled entries against
    the oracle quadrature, and properties of the posterior after 2 sweeps."""
    cat = make_catalogue("c2_plain_20k", truth="mean")
    with init(gm, cat, precision=gm.PREC_FP32, cg_tol=1e-6) as ctx:
        nnz = ctx.build_cov()
        i, j, v = csr_external(ctx)
        m0, kd = ctx.get_prior()
        ctx.ep_sweep(2)
        mu, var = ctx.get_posterior()
        st = ctx.stats()
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * cat["s"][:, None]
    pairs = O.neighbour_pairs(x, cat["cutoff_pc"])
    assert nnz == 20000 + 2 * len(pairs)
    key_gpu = np.sort(i.astype(np.int64) * 20000 + j)
    kp = np.concatenate([pairs[:, 0] * 20000 + pairs[:, 1], pairs[:, 1] * 20000 + pairs[:, 0],
                         np.arange(20000) * 20001])
    np.testing.assert_array_equal(key_gpu, np.sort(kp))
    rng = np.random.default_rng(1)
    pick = rng.choice(len(i), 300, replace=False)
    ii, jj = i[pick], j[pick]
    g = lambda r: O.g_of_r(r, 1.0, 20.0)  # noqa: E731
    R = O.pair_R(cat["s"][ii], cat["s"][jj], ((u[ii] - u[jj]) ** 2).sum(1), g, 64)
    d = np.sqrt(((x[ii] - x[jj]) ** 2).sum(1))
    ref = np.log1p(R) * O.wendland(d / cat["cutoff_pc"])
    np.testing.assert_allclose(v[pick], ref, rtol=2e-5, atol=1e-9)
    assert np.all(np.isfinite(mu)) and np.all(var > 0)
    assert np.all(var <= kd * (1 + 1e-5))
    assert st["cg_resid_mean"] <= 1e-6 * 1.01
    # updates with a negative site precision are skipped: only stars with
    # weak positive observations (non-log-concave likelihood) can do this
    assert st["sites_skipped"] < 0.01 * 20000
