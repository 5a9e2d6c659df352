"""The allocation-free site update (gm_site_update_noalloc) against the
context path.

Callers that cannot allocate device memory while they run (a framework that
owns all device memory through its own pool, a process inside a fixed memory
budget, a latency-bound service loop) use the allocation-free entry point on
arrays they own.  This test drives it through the C ABI on device arrays and
checks, on two calls in a row, that it produces the same sites as the sweep
of a context (gm_ep_sweep) started from the same state.
"""
import ctypes as C

import numpy as np
import pytest

from synth import make_catalogue

pytestmark = pytest.mark.gpu


def test_noalloc_site_update_matches_context_sweep():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as gm
    L = gm.lib()
    dev = torch.device("cuda:0")
    cat = make_catalogue("c1_plain_400")
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP64, warm_start=0)
    obs = torch.tensor(cat["A_obs"], dtype=torch.float64, device=dev)
    sig = torch.tensor(cat["A_sigma"], dtype=torch.float64, device=dev)
    n = len(cat["s"])
    stream = torch.cuda.current_stream(dev).cuda_stream
    with gm.ep_init(cfg, cat["l"], cat["b"], cat["s"], cat["A_obs"], cat["A_sigma"]) as ctx:
        ctx.build_cov()
        ctx.ep_sweep(2)
        for call in range(2):
            # state before the next sweep, in caller order, on the device
            mu = torch.empty(n, dtype=torch.float64, device=dev)
            var = torch.empty(n, dtype=torch.float64, device=dev)
            tau = torch.empty(n, dtype=torch.float64, device=dev)
            nu = torch.empty(n, dtype=torch.float64, device=dev)
            ctx.get_posterior(out=(mu, var))
            ctx.get_sites(out=(tau, nu))
            torch.cuda.synchronize()
            delta, skipped = C.c_double(-1.0), C.c_int64(-1)
            st = L.gm_site_update_noalloc(n, mu.data_ptr(), var.data_ptr(), obs.data_ptr(),
                                          sig.data_ptr(), tau.data_ptr(), nu.data_ptr(),
                                          cfg.likelihood, cfg.damping, cfg.vc_floor,
                                          C.c_void_p(stream), C.byref(delta), C.byref(skipped))
            assert st == 0, L.gm_status_str(st)
            done, ctx_delta = ctx.ep_sweep(1)
            t_ref, n_ref = ctx.get_sites()
            np.testing.assert_allclose(tau.cpu().numpy(), t_ref, rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(nu.cpu().numpy(), n_ref, rtol=1e-12, atol=1e-12)
            assert skipped.value == ctx.stats()["sites_skipped"]
            assert delta.value == pytest.approx(ctx_delta, rel=1e-12, abs=1e-15)
    # sizes beyond the scratch capacity and host pointers are rejected
    big = L.gm_site_update_noalloc(1_048_577, mu.data_ptr(), var.data_ptr(), obs.data_ptr(),
                                   sig.data_ptr(), tau.data_ptr(), nu.data_ptr(), 0, 1.0, 1e-8,
                                   None, None, None)
    assert big == 1
    host = np.zeros(n)
    st = L.gm_site_update_noalloc(n, host.ctypes.data, var.data_ptr(), obs.data_ptr(),
                                  sig.data_ptr(), tau.data_ptr(), nu.data_ptr(), 0, 1.0, 1e-8,
                                  None, None, None)
    assert st == 1
