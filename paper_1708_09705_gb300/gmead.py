"""Python binding of libgmead (argument marshalling only).

Every computation runs in the CUDA library; this module converts arrays to
pointers, routes device allocations to PyTorch's caching allocator and turns
status codes into exceptions.  The names follow the C ABI in include/gmead.h:
ep_init, build_cov, ep_sweep, predict, get_posterior, get_sites, set_sites.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
they must be contiguous float64 (int64 for permutations).  Outputs are
returned as numpy arrays unless CUDA tensors are passed as `out`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmead.so")

PREC_FP64, PREC_FP32 = 0, 1
FORM_LOGNORMAL, FORM_LINEAR = 0, 1
TAPER_WENDLAND, TAPER_HARD = 0, 1
LIK_GAUSS_IN_A, LIK_GAUSS_IN_LNA = 0, 1
COV_QUADRATURE, COV_SURROGATE = 0, 1
QUAD_GL, QUAD_BAND = 0, 1

STATUS = {0: "GM_OK", 1: "GM_E_INVAL", 2: "GM_E_NOMEM", 3: "GM_E_CUDA", 4: "GM_E_NOT_SPD",
          5: "GM_E_NOCONV", 6: "GM_E_NONFINITE", 7: "GM_E_TIMEOUT", 8: "GM_E_STATE"}

# every symbol include/gmead.h declares
EXPORTS = ["gm_config_default", "gm_ep_init", "gm_ep_init_fields", "gm_build_cov", "gm_ep_sweep", "gm_predict",
           "gm_get_posterior", "gm_get_sites", "gm_set_sites", "gm_get_prior", "gm_get_perm",
           "gm_get_csr", "gm_get_stats", "gm_stream", "gm_status_str", "gm_last_error",
           "gm_destroy", "gm_profile", "gm_kernel_time_count", "gm_kernel_time",
           "gm_site_update_noalloc", "gm_surrogate_param_count", "gm_surrogate_set_params",
           "gm_surrogate_get_params", "gm_surrogate_eval", "gm_surrogate_train",
           "gm_surrogate_grad", "gm_get_probe_colours", "gm_get_entries", "gm_predict_pairs",
           "gm_predict_sightlines", "gm_monotone_sample", "gm_pic_posterior",
           "gm_pic_predict", "gm_set_mean_fn", "gm_learn_mean", "gm_cov_rows"]


class GmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("outer_scale_pc", C.c_double), ("rho_bar", C.c_double),
                ("cutoff_pc", C.c_double), ("n_nodes", C.c_int32), ("form", C.c_int32),
                ("taper", C.c_int32), ("precision", C.c_int32), ("likelihood", C.c_int32),
                ("cg_max_iter", C.c_int32), ("damping", C.c_double), ("vc_floor", C.c_double),
                ("cg_tol", C.c_double), ("rhs_panel", C.c_int32), ("warm_start", C.c_int32),
                ("cov_source", C.c_int32), ("deflate", C.c_int32),
                ("surrogate_gate", C.c_double), ("probe_factor", C.c_double),
                ("quad_rule", C.c_int32), ("tc_products", C.c_int32)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("n_stars", C.c_int64), ("nnz", C.c_int64), ("n_pairs", C.c_int64),
                ("cg_iters_mean", C.c_int64), ("cg_iters_var", C.c_int64),
                ("sites_skipped", C.c_int64), ("kernel_launches", C.c_int64),
                ("last_max_delta", C.c_double), ("cg_resid_mean", C.c_double),
                ("cg_resid_var", C.c_double), ("surrogate_fallback", C.c_int64),
                ("surrogate_loss", C.c_double), ("surrogate_val_rmse", C.c_double),
                ("surrogate_gate_frac", C.c_double), ("probe_colours", C.c_int64),
                ("tile_ksteps", C.c_int64), ("variance_panel_width", C.c_int64),
                ("tile_variant", C.c_int64)]


_lib = None


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.gm_config_default.argtypes = [C.POINTER(Config)]
        L.gm_config_default.restype = None
        L.gm_ep_init.argtypes = [C.POINTER(vp), C.POINTER(Config), i64, vp, vp, vp, vp, vp, vp,
                                 C.POINTER(Allocator)]
        L.gm_ep_init_fields.argtypes = [C.POINTER(vp), C.POINTER(Config), i64, vp, vp, vp, vp, vp,
                                        i32, vp, vp, vp, vp, C.POINTER(Allocator)]
        L.gm_build_cov.argtypes = [vp, C.POINTER(i64)]
        L.gm_ep_sweep.argtypes = [vp, i32, dbl, C.POINTER(i32), C.POINTER(dbl)]
        L.gm_predict.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        for f in ("gm_get_posterior", "gm_get_sites", "gm_set_sites", "gm_get_prior"):
            getattr(L, f).argtypes = [vp, vp, vp]
        L.gm_get_perm.argtypes = [vp, vp]
        L.gm_get_probe_colours.argtypes = [vp, vp]
        L.gm_get_entries.argtypes = [vp, i64, vp, vp, vp]
        L.gm_predict_pairs.argtypes = [vp, i64, vp, vp, vp, dbl, vp, vp, vp]
        L.gm_predict_sightlines.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp]
        L.gm_monotone_sample.argtypes = [vp, i64, i32, vp, vp, vp, i32, i32, vp, vp]
        L.gm_pic_posterior.argtypes = [vp, i32, vp, i64, vp, vp, vp, vp, vp]
        L.gm_pic_predict.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        L.gm_get_csr.argtypes = [vp, vp, vp, vp]
        L.gm_set_mean_fn.argtypes = [vp, vp, dbl, dbl]
        L.gm_cov_rows.argtypes = [vp, i64, i64, i32, i64, vp, vp, vp, C.POINTER(i64),
                                  C.POINTER(i64)]
        L.gm_learn_mean.argtypes = [vp, vp, vp, vp, dbl, dbl, i32, dbl, vp, vp,
                                    C.POINTER(dbl), C.POINTER(i32)]
        L.gm_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.gm_stream.argtypes = [vp]
        L.gm_stream.restype = vp
        L.gm_status_str.argtypes = [C.c_int]
        L.gm_status_str.restype = C.c_char_p
        L.gm_last_error.argtypes = [vp]
        L.gm_last_error.restype = C.c_char_p
        L.gm_destroy.argtypes = [vp]
        L.gm_destroy.restype = None
        L.gm_profile.argtypes = [vp, i32]
        L.gm_surrogate_param_count.argtypes = []
        L.gm_surrogate_param_count.restype = i64
        L.gm_surrogate_set_params.argtypes = [vp, vp, i64]
        L.gm_surrogate_get_params.argtypes = [vp, vp, i64]
        L.gm_surrogate_eval.argtypes = [vp, i64, vp, vp, vp, dbl, dbl, vp, vp]
        L.gm_surrogate_train.argtypes = [vp, i64, i32, i32, dbl, C.c_uint64]
        L.gm_surrogate_grad.argtypes = [vp, i64, vp, vp, dbl, vp, C.POINTER(dbl)]
        L.gm_site_update_noalloc.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, dbl, dbl, vp,
                                             C.POINTER(dbl), C.POINTER(i64)]
        L.gm_site_update_noalloc.restype = C.c_int
        L.gm_kernel_time_count.argtypes = [vp]
        L.gm_kernel_time_count.restype = i32
        L.gm_kernel_time.argtypes = [vp, i32, C.POINTER(C.c_char_p), C.POINTER(i64),
                                     C.POINTER(dbl)]
        for f in ("gm_ep_init", "gm_ep_init_fields", "gm_build_cov", "gm_ep_sweep", "gm_predict", "gm_get_posterior",
                  "gm_get_sites", "gm_set_sites", "gm_get_prior", "gm_get_perm", "gm_get_csr",
                  "gm_get_stats", "gm_profile", "gm_kernel_time", "gm_surrogate_set_params",
                  "gm_surrogate_get_params", "gm_surrogate_eval", "gm_surrogate_train",
                  "gm_surrogate_grad", "gm_get_probe_colours", "gm_get_entries",
                  "gm_predict_pairs", "gm_set_mean_fn", "gm_learn_mean", "gm_cov_rows"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def default_config(**kw) -> Config:
    cfg = Config()
    lib().gm_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _ptr(a, dtype=np.float64):
    """(pointer, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        want = torch.float64 if dtype == np.float64 else (
            torch.int64 if dtype == np.int64 else torch.int32)
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


def _torch_allocator(device_index):
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=device_index,
                                                          stream=int(stream or 0)))
        except Exception:  # out of memory -> the library reports GM_E_NOMEM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    return Allocator(fa, ff, None), (fa, ff)


def _ptr_any(a):
    """Raw address of a contiguous numpy array or torch tensor (no copy)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise TypeError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise TypeError("array must be contiguous")
    return a.ctypes.data


class Context:
    """Owns one gm_ctx.  Created by ep_init."""

    def __init__(self, handle, n, keep, cfg=None):
        self._h = handle
        self.n = int(n)
        self._keep = keep
        self.precision = cfg.precision if cfg is not None else PREC_FP64
        self.cfg_source = cfg.cov_source if cfg is not None else COV_QUADRATURE

    def _check(self, st):
        if st != 0:
            msg = lib().gm_last_error(self._h).decode()
            raise GmError(st, msg)

    # ---- hot path
    def build_cov(self) -> int:
        nnz = C.c_int64(0)
        self._check(lib().gm_build_cov(self._h, C.byref(nnz)))
        return nnz.value

    def ep_sweep(self, n_sweeps=1, tol=0.0):
        done, delta = C.c_int32(0), C.c_double(0)
        self._check(lib().gm_ep_sweep(self._h, int(n_sweeps), float(tol), C.byref(done),
                                      C.byref(delta)))
        return done.value, delta.value

    def predict(self, l, b, s, out=None):
        pl, kl = _ptr(l)
        pb, kb = _ptr(b)
        ps, ks = _ptr(s)
        nq = len(kl) if hasattr(kl, "__len__") else int(kl.numel())
        mean, var = out if out is not None else (np.empty(nq), np.empty(nq))
        pm, km = _ptr(mean)
        pv, kv = _ptr(var)
        self._check(lib().gm_predict(self._h, nq, pl, pb, ps, pm, pv))
        return mean, var

    def predict_pairs(self, l, b, s, ds=10.0):
        """Joint predictive at s and s + ds per query and the pseudo-density
        moments: (means (nq, 2), covariances (nq, 3), density (nq, 2))."""
        l, b, s = (np.ascontiguousarray(v, dtype=np.float64) for v in (l, b, s))
        nq = len(s)
        mean, cov, dens = np.empty((nq, 2)), np.empty((nq, 3)), np.empty((nq, 2))
        self._check(lib().gm_predict_pairs(self._h, nq, l.ctypes.data, b.ctypes.data,
                                           s.ctypes.data, float(ds), mean.ctypes.data,
                                           cov.ctypes.data, dens.ctypes.data))
        return mean, cov, dens

    def predict_sightlines(self, l, b, s):
        """Joint predictive of the m points s[q, :] (increasing) on each
        sightline (l[q], b[q]): (means (nsl, m), covariances (nsl, m, m))."""
        l, b = (np.ascontiguousarray(v, dtype=np.float64) for v in (l, b))
        s = np.ascontiguousarray(np.atleast_2d(s), dtype=np.float64)
        nsl, m = s.shape
        mean, cov = np.empty((nsl, m)), np.empty((nsl, m, m))
        self._check(lib().gm_predict_sightlines(self._h, nsl, m, l.ctypes.data, b.ctypes.data,
                                                s.ctypes.data, mean.ctypes.data,
                                                cov.ctypes.data))
        return mean, cov

    def monotone_sample(self, mean, cov, momenta, n_burn):
        """Exact-HMC samples of N(mean[q], cov[q]) truncated to a
        non-decreasing sequence; momenta: (nsl, n_burn + n_samples, m)
        standard normal draws.  Returns (samples (nsl, n_samples, m), wall
        hits (nsl,))."""
        mean = np.ascontiguousarray(np.atleast_2d(mean), dtype=np.float64)
        nsl, m = mean.shape
        cov = np.ascontiguousarray(cov, dtype=np.float64).reshape(nsl, m, m)
        momenta = np.ascontiguousarray(momenta, dtype=np.float64)
        T = momenta.shape[1]
        assert momenta.shape == (nsl, T, m) and 0 <= n_burn <= T
        ns = T - int(n_burn)
        out, hits = np.empty((nsl, ns, m)), np.empty(nsl, dtype=np.int64)
        self._check(lib().gm_monotone_sample(self._h, nsl, m, mean.ctypes.data, cov.ctypes.data,
                                             momenta.ctypes.data, int(n_burn), ns,
                                             out.ctypes.data, hits.ctypes.data))
        return out, hits

    def pic_posterior(self, block_of, l, b, s):
        """PITC / PIC posterior of ln A at the inducing points (l, b, s) with
        the stars split into sub-catalogues block_of (caller order):
        (mean (R,), covariance (R, R))."""
        blk = np.ascontiguousarray(block_of, dtype=np.int32)
        l, b, s = (np.ascontiguousarray(v, dtype=np.float64) for v in (l, b, s))
        R = len(s)
        mean, cov = np.empty(R), np.empty((R, R))
        self._check(lib().gm_pic_posterior(self._h, int(blk.max()) + 1, blk.ctypes.data, R,
                                           l.ctypes.data, b.ctypes.data, s.ctypes.data,
                                           mean.ctypes.data, cov.ctypes.data))
        return mean, cov

    def pic_predict(self, q_block, l, b, s):
        """PIC predictive (mean, var) at queries (l, b, s) assigned to the
        sub-catalogues q_block, after pic_posterior."""
        qb = np.ascontiguousarray(q_block, dtype=np.int32)
        l, b, s = (np.ascontiguousarray(v, dtype=np.float64) for v in (l, b, s))
        nq = len(s)
        mean, var = np.empty(nq), np.empty(nq)
        self._check(lib().gm_pic_predict(self._h, nq, qb.ctypes.data, l.ctypes.data,
                                         b.ctypes.data, s.ctypes.data, mean.ctypes.data,
                                         var.ctypes.data))
        return mean, var

    # ---- mean function of the density and its hyperparameters (Sect. 5)
    def set_mean_fn(self, theta, r_sun_pc=8000.0, bump_width_pc=400.0):
        """Disc + bump mean density theta = (L, H, rho0, s_bump, A_bump), or
        None for the constant mean density."""
        t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        self._check(lib().gm_set_mean_fn(self._h, None if t is None else t.ctypes.data,
                                         float(r_sun_pc), float(bump_width_pc)))

    def learn_mean(self, theta0, prior_mean, prior_sd=None, r_sun_pc=8000.0,
                   bump_width_pc=400.0, max_iter=50, tol=1e-10):
        """Mode and Laplace covariance (of ln theta) of the five mean-function
        hyperparameters; returns dict(theta, cov_phi, log_post, iters)."""
        t0 = np.ascontiguousarray(theta0, dtype=np.float64)
        pm = np.ascontiguousarray(prior_mean, dtype=np.float64)
        ps = pm.copy() if prior_sd is None else np.ascontiguousarray(prior_sd, dtype=np.float64)
        th, cov = np.empty(5), np.empty((5, 5))
        lp, it = C.c_double(0.0), C.c_int32(0)
        self._check(lib().gm_learn_mean(self._h, t0.ctypes.data, pm.ctypes.data, ps.ctypes.data,
                                        float(r_sun_pc), float(bump_width_pc), int(max_iter),
                                        float(tol), th.ctypes.data, cov.ctypes.data,
                                        C.byref(lp), C.byref(it)))
        return dict(theta=th, cov_phi=cov, log_post=lp.value, iters=it.value)

    def cov_rows(self, row0, nrows, source=None, out=None):
        """Covariance rows row0 .. row0 + nrows - 1 (internal order) assembled
        without a stored matrix; returns (row_ptr, col, val, fallback).  out:
        optional (col, val) arrays (numpy or torch, host or device) with room."""
        src = self.cfg_source if source is None else source
        rp = np.empty(nrows + 1, dtype=np.int64)
        nnz, fb = C.c_int64(0), C.c_int64(0)
        if out is None:
            st = lib().gm_cov_rows(self._h, int(row0), int(nrows), int(src), 0, rp.ctypes.data,
                                   None, None, C.byref(nnz), C.byref(fb))
            if st not in (0, 1):
                self._check(st)
            vdt = np.float32 if self.precision == PREC_FP32 else np.float64
            col = np.empty(max(nnz.value, 1), dtype=np.int32)
            val = np.empty(max(nnz.value, 1), dtype=vdt)
            cap = nnz.value
        else:
            col, val = out
            cap = col.numel() if hasattr(col, "numel") else col.size
        self._check(lib().gm_cov_rows(self._h, int(row0), int(nrows), int(src), int(cap),
                                      rp.ctypes.data, _ptr_any(col), _ptr_any(val),
                                      C.byref(nnz), C.byref(fb)))
        return rp, col[:nnz.value], val[:nnz.value], fb.value

    # ---- state
    def _pair_out(self, fn, out):
        a, b = out if out is not None else (np.empty(self.n), np.empty(self.n))
        pa, ka = _ptr(a)
        pb, kb = _ptr(b)
        self._check(fn(self._h, pa, pb))
        return a, b

    def get_posterior(self, out=None):
        return self._pair_out(lib().gm_get_posterior, out)

    def get_sites(self, out=None):
        return self._pair_out(lib().gm_get_sites, out)

    def get_prior(self, out=None):
        return self._pair_out(lib().gm_get_prior, out)

    def set_sites(self, tau, nu):
        pt, kt = _ptr(tau)
        pn, kn = _ptr(nu)
        self._check(lib().gm_set_sites(self._h, pt, pn))

    def get_perm(self):
        out = np.empty(self.n, dtype=np.int64)
        self._check(lib().gm_get_perm(self._h, out.ctypes.data))
        return out

    def get_entries(self, i, j):
        """Stored K_ij for caller index pairs (0 beyond the cutoff)."""
        i = np.ascontiguousarray(i, dtype=np.int64)
        j = np.ascontiguousarray(j, dtype=np.int64)
        out = np.empty(len(i), dtype=np.float64)
        self._check(lib().gm_get_entries(self._h, len(i), i.ctypes.data, j.ctypes.data,
                                         out.ctypes.data))
        return out

    def get_probe_colours(self):
        """Colour class of each star (caller order) when probing is on."""
        out = np.empty(self.n, dtype=np.int32)
        self._check(lib().gm_get_probe_colours(self._h, out.ctypes.data))
        return out

    def get_csr(self):
        nnz = self.stats()["nnz"]
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        val = np.empty(max(nnz, 1), dtype=np.float64)
        self._check(lib().gm_get_csr(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col[:nnz], val[:nnz]

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().gm_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def profile(self, enable=True):
        """Per-kernel CUDA-event timing on the context stream (gm_profile)."""
        self._check(lib().gm_profile(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{kernel name: (launches, total ms)} accumulated since profile(True)."""
        out = {}
        for k in range(lib().gm_kernel_time_count(self._h)):
            name, cnt, ms = C.c_char_p(), C.c_int64(), C.c_double()
            self._check(lib().gm_kernel_time(self._h, k, C.byref(name), C.byref(cnt),
                                             C.byref(ms)))
            out[name.value.decode()] = (cnt.value, ms.value)
        return out

    # ---- covariance surrogate
    def surrogate_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(lib().gm_surrogate_set_params(self._h, p.ctypes.data, p.size))

    def surrogate_get_params(self):
        out = np.empty(lib().gm_surrogate_param_count(), dtype=np.float32)
        self._check(lib().gm_surrogate_get_params(self._h, out.ctypes.data, out.size))
        return out

    def surrogate_eval(self, si, sj, chord, sigma2, L0):
        a, ka = _ptr(si)
        b, kb = _ptr(sj)
        c, kc = _ptr(chord)
        n = len(ka)
        y = np.empty(n, dtype=np.float32)
        e = np.empty(n, dtype=np.float32)
        self._check(lib().gm_surrogate_eval(self._h, n, a, b, c, float(sigma2), float(L0),
                                            y.ctypes.data, e.ctypes.data))
        return y, e

    def surrogate_train(self, n_pairs=1_000_000, steps=4000, batch=8192, lr=2e-3, seed=1):
        self._check(lib().gm_surrogate_train(self._h, int(n_pairs), int(steps), int(batch),
                                             float(lr), int(seed)))
        return self.stats()

    def surrogate_grad(self, X, Y, lam):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.empty(lib().gm_surrogate_param_count(), dtype=np.float32)
        loss = C.c_double()
        self._check(lib().gm_surrogate_grad(self._h, len(Y), X.ctypes.data, Y.ctypes.data,
                                            float(lam), g.ctypes.data, C.byref(loss)))
        return loss.value, g

    @property
    def stream(self) -> int:
        return lib().gm_stream(self._h) or 0

    def close(self):
        if self._h:
            lib().gm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ep_init(cfg: Config, l, b, s, obs, obs_sigma, stream=None, torch_alloc=True,
            field_id=None, field_L0=None, field_cutoff=None) -> Context:
    """Create a context (gm_ep_init, or gm_ep_init_fields when field_id is
    given).  `stream` is a cudaStream_t as int, a torch.cuda.Stream, or None
    for torch's current stream when torch is loaded.  With torch_alloc,
    device memory comes from torch's caching allocator."""
    L = lib()
    keep = []
    ptrs = []
    n = None
    for a in (l, b, s, obs, obs_sigma):
        p, k = _ptr(a)
        keep.append(k)
        ptrs.append(p)
        m = len(k) if hasattr(k, "__len__") else int(k.numel())
        if n is None:
            n = m
        elif m != n:
            raise ValueError("input arrays differ in length")
    alloc_ptr = None
    sptr = 0
    try:
        import torch
        if torch.cuda.is_available():
            dev = torch.cuda.current_device()
            if stream is None:
                sptr = torch.cuda.current_stream(dev).cuda_stream
            elif hasattr(stream, "cuda_stream"):
                sptr = stream.cuda_stream
            else:
                sptr = int(stream)
            if torch_alloc:
                alloc, fns = _torch_allocator(dev)
                keep += [alloc, fns]
                alloc_ptr = C.byref(alloc)
    except ImportError:
        sptr = int(stream or 0)
    h = C.c_void_p()
    if field_id is None:
        st = L.gm_ep_init(C.byref(h), C.byref(cfg), int(n), *ptrs, C.c_void_p(sptr), alloc_ptr)
    else:
        fid = np.ascontiguousarray(field_id, dtype=np.int32)
        nf = int(fid.max()) + 1 if field_L0 is None else len(field_L0)
        fL0 = None if field_L0 is None else np.ascontiguousarray(field_L0, dtype=np.float64)
        fct = None if field_cutoff is None else np.ascontiguousarray(field_cutoff, dtype=np.float64)
        keep += [fid, fL0, fct]
        st = L.gm_ep_init_fields(C.byref(h), C.byref(cfg), int(n), *ptrs, nf, fid.ctypes.data,
                                 None if fL0 is None else fL0.ctypes.data,
                                 None if fct is None else fct.ctypes.data, C.c_void_p(sptr),
                                 alloc_ptr)
    ctx = Context(h, n, keep, cfg)
    if st != 0:
        msg = L.gm_last_error(h).decode() if h else STATUS.get(st, str(st))
        ctx.close()
        raise GmError(st, msg)
    return ctx


# module-level names matching the C ABI
def build_cov(ctx: Context) -> int:
    return ctx.build_cov()


def ep_sweep(ctx: Context, n_sweeps=1, tol=0.0):
    return ctx.ep_sweep(n_sweeps, tol)


def predict(ctx: Context, l, b, s, out=None):
    return ctx.predict(l, b, s, out)


def get_posterior(ctx: Context, out=None):
    return ctx.get_posterior(out)


def config_from_catalogue(cat, **kw) -> Config:
    """Config with the hyperparameters of a synthetic catalogue dict; the
    node rule is the workload's: n_nodes Gauss-Legendre nodes per sightline."""
    base = dict(sigma2=float(cat["sigma2"]), outer_scale_pc=float(cat["outer_scale_pc"]),
                rho_bar=float(cat["rho_bar"]), cutoff_pc=float(cat["cutoff_pc"]),
                n_nodes=int(cat["n_nodes"]), quad_rule=QUAD_GL)
    base.update(kw)
    return default_config(**base)
