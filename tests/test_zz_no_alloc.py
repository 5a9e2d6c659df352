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


def _compare_with_context(side_stream: bool):
    """Two allocation-free updates in a row against two context sweeps; with
    side_stream the calls run on a non-blocking torch stream."""
    import torch
    import paper_1708_09705_gb300 as gm
    L = gm.lib()
    dev = torch.device("cuda:0")
    cat = make_catalogue("c1_plain_400")
    cfg = gm.config_from_catalogue(cat, precision=gm.PREC_FP64, warm_start=0)
    obs = torch.tensor(cat["A_obs"], dtype=torch.float64, device=dev)
    sig = torch.tensor(cat["A_sigma"], dtype=torch.float64, device=dev)
    n = len(cat["s"])
    side = torch.cuda.Stream(dev) if side_stream else None
    stream = (side if side_stream else torch.cuda.current_stream(dev)).cuda_stream
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
    return L, n, (mu, var, obs, sig, tau, nu)


def _gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as gm
    return gm


def test_noalloc_site_update_matches_context_sweep():
    _gm()
    L, n, (mu, var, obs, sig, tau, nu) = _compare_with_context(False)
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


def test_noalloc_first_call_on_a_side_stream_in_a_fresh_process():
    """The first call of a process uploads the quadrature rule; a kernel on a
    non-blocking stream must still see it."""
    import os
    import subprocess
    import sys
    _gm()
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_zz_no_alloc as t; "
            "t._compare_with_context(True); print('ok')" % (os.path.dirname(here), here))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_noalloc_rejects_memory_of_another_gpu():
    torch = pytest.importorskip("torch")
    gm = _gm()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    L = gm.lib()
    n = 64
    torch.cuda.set_device(0)
    mine = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(6)]
    other = torch.zeros(n, dtype=torch.float64, device="cuda:1")
    st = L.gm_site_update_noalloc(n, other.data_ptr(), *[t.data_ptr() for t in mine[1:]],
                                  0, 1.0, 1e-8, None, None, None)
    assert st == 1
