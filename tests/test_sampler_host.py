"""The sightline sampler's per-sightline routine (csrc/gm_hmc.cuh, run by the
device kernel one thread per sightline) compiled for the host and checked
against the oracle's exact HMC (oracle/monotone.py) with the same momenta.
This checks the arithmetic and the strided layout without a GPU; the device
run itself is checked in test_gpu_sightline.py.  CPU only."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import monotone as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1708_09705_gb300", "csrc")

# Stages the caller layout into the sightline-fastest layout the kernel uses
# (the mapping of k_sl_stage) and runs one sightline after another.
HARNESS = r"""
#include "gm_hmc.cuh"
#include <vector>
extern "C" unsigned hmc_host(int64_t nsl, int m, const double* mean, const double* cov,
                             const double* mom, int n_burn, int n_samples, double* out,
                             int64_t* hits) {
  std::vector<double> mu_t(m * nsl), S_t((size_t)m * m * nsl), L_t((size_t)m * m * nsl),
      y_t(m * nsl), w_t(m * nsl);
  for (int64_t q = 0; q < nsl; ++q) {
    for (int i = 0; i < m; ++i) mu_t[i * nsl + q] = mean[q * m + i];
    for (int e = 0; e < m * m; ++e) S_t[e * nsl + q] = cov[q * m * m + e];
  }
  const int64_t T = n_burn + n_samples;
  unsigned st = 0;
  for (int64_t q = 0; q < nsl; ++q)
    st |= gmhmc::sample_sightline(&mu_t[q], &S_t[q], &L_t[q], &y_t[q], &w_t[q], nsl,
                                  mom + q * T * m, out + q * (int64_t)n_samples * m, m,
                                  n_burn, n_samples, &hits[q]);
  return st;
}
// the warp kernel's phase sequence, its 32 lanes run one after another
// between the warp barriers
extern "C" unsigned hmc_warp_host(int64_t nsl, int m, const double* mean, const double* cov,
                                  const double* mom, int n_burn, int n_samples, double* out,
                                  int64_t* hits) {
  std::vector<double> mu_t(m * nsl), S_t((size_t)m * m * nsl), SL(2 * m * m);
  for (int64_t q = 0; q < nsl; ++q) {
    for (int i = 0; i < m; ++i) mu_t[i * nsl + q] = mean[q * m + i];
    for (int e = 0; e < m * m; ++e) S_t[e * nsl + q] = cov[q * m * m + e];
  }
  const int64_t T = n_burn + n_samples;
  unsigned flags = 0;
  for (int64_t q = 0; q < nsl; ++q) {
    gmhmc::WarpState W;
    W.S = SL.data();
    W.L = SL.data() + m * m;
    for (int l = 0; l < 32; ++l) gmhmc::w_stage(W, l, m, &mu_t[q], &S_t[q], nsl);
    gmhmc::w_setup(W, m);
    double* o = out + q * (int64_t)n_samples * m;
    if (W.status) {
      for (int64_t k = 0; k < (int64_t)n_samples * m; ++k) o[k] = NAN;
      hits[q] = 0;
      flags |= 1u;
      continue;
    }
    for (int64_t it = 0; it < T; ++it) {
      for (int l = 0; l < 32; ++l) gmhmc::w_momentum(W, l, m, mom + (q * T + it) * m);
      for (int l = 0; l < 32; ++l) gmhmc::w_velocity(W, l, m);
      W.t_left = gmhmc::kHalfPi;
      int n = 0;
      for (; n < gmhmc::kMaxWallHits; ++n) {
        for (int l = 0; l < 32; ++l) gmhmc::w_hit(W, l, m);
        double tb;
        const int j = gmhmc::w_best(W, m, &tb);
        if (j < 0) {
          const double tl = W.t_left;
          for (int l = 0; l < 32; ++l) gmhmc::w_rotate(W, l, m, tl);
          break;
        }
        for (int l = 0; l < 32; ++l) gmhmc::w_rotate(W, l, m, tb);
        gmhmc::w_reflect_factor(W, m, j);
        for (int l = 0; l < 32; ++l) gmhmc::w_reflect(W, l, m, j);
        W.t_left -= tb;
        W.nhits++;
      }
      if (n == gmhmc::kMaxWallHits) flags |= 2u;
      if (it >= n_burn)
        for (int l = 0; l < m; ++l) o[(it - n_burn) * m + l] = W.mu[l] + W.y[l];
    }
    hits[q] = W.nhits;
  }
  return flags;
}
"""


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("hmc")
    src, so = d / "harness.cpp", d / "libhmc_host.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                    f"-I{CSRC}", str(src), "-o", str(so)], check=True)
    L = C.CDLL(str(so))
    vp = C.c_void_p
    L.hmc_host.argtypes = [C.c_int64, C.c_int, vp, vp, vp, C.c_int, C.c_int, vp, vp]
    L.hmc_host.restype = C.c_uint
    L.hmc_warp_host.argtypes = L.hmc_host.argtypes
    L.hmc_warp_host.restype = C.c_uint
    return L


def run(L, mu, S, mom, burn, warp=False):
    nsl, m = mu.shape
    ns = mom.shape[1] - burn
    out = np.zeros((nsl, ns, m))
    hits = np.zeros(nsl, np.int64)
    mu, S, mom = (np.ascontiguousarray(a, dtype=np.float64) for a in (mu, S, mom))
    fn = L.hmc_warp_host if warp else L.hmc_host
    st = fn(nsl, m, mu.ctypes.data, S.ctypes.data, mom.ctypes.data, burn, ns,
            out.ctypes.data, hits.ctypes.data)
    return st, out, hits


def sightlines(rng, nsl, m, drift=0.0):
    s = np.linspace(0.0, 1.0, m)
    mu, S = [], []
    for _ in range(nsl):
        S.append((0.02 + 0.03 * rng.random()) * np.exp(-np.abs(s[:, None] - s[None, :]) / 0.4)
                 + 1e-4 * np.eye(m))
        mu.append(np.cumsum(rng.normal(drift, 0.05, m)) - 1.0)
    return np.array(mu), np.array(S)


@pytest.mark.parametrize("m", [2, 6, 17])
def test_host_build_matches_oracle_chain(host_lib, m):
    rng = np.random.default_rng(m)
    nsl, burn, ns = 12, 8, 30
    mu, S = sightlines(rng, nsl, m)
    mom = rng.standard_normal((nsl, burn + ns, m))
    st, out, hits = run(host_lib, mu, S, mom, burn)
    assert st == 0
    assert hits.sum() > 10 * nsl           # the walls bind: the mean often decreases
    ref = np.array([M.monotone_sightline(mu[q], S[q], ns, None, burn=burn, momenta=mom[q])
                    for q in range(nsl)])
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)
    assert np.all(np.diff(out, axis=2) >= 0)


def test_single_point_has_no_walls(host_lib):
    """m = 1: the step is the exact rotation y cos(pi/2) + w sin(pi/2) = w,
    so each sample is mu + sd * momentum."""
    mu = np.array([[0.3], [-1.2]])
    S = np.array([[[0.25]], [[4.0]]])
    mom = np.random.default_rng(1).standard_normal((2, 6, 1))
    st, out, hits = run(host_lib, mu, S, mom, 1)
    assert st == 0 and np.all(hits == 0)
    np.testing.assert_allclose(out[:, :, 0], mu + np.sqrt(S[:, :, 0]) * mom[:, 1:, 0],
                               atol=1e-15)


def test_not_positive_definite_gives_nan_and_status(host_lib):
    mu = np.zeros((2, 2))
    S = np.array([np.eye(2), [[1.0, 2.0], [2.0, 1.0]]])
    mom = np.ones((2, 3, 2))
    st, out, _ = run(host_lib, mu, S, mom, 1)
    assert st == 1
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1]))


@pytest.mark.parametrize("m", [2, 9, 32])
def test_warp_phases_give_the_thread_chain(host_lib, m):
    """The warp kernel's phases (one lane per point) run lane by lane give the
    one-thread chain and the oracle's chain, wall hits included."""
    rng = np.random.default_rng(40 + m)
    nsl, burn, ns = 6, 5, 20
    mu, S = sightlines(rng, nsl, m)
    mom = rng.standard_normal((nsl, burn + ns, m))
    st_t, out_t, hits_t = run(host_lib, mu, S, mom, burn)
    st_w, out_w, hits_w = run(host_lib, mu, S, mom, burn, warp=True)
    assert st_t == st_w == 0
    np.testing.assert_array_equal(hits_w, hits_t)
    np.testing.assert_allclose(out_w, out_t, rtol=0, atol=1e-13)
    ref = np.array([M.monotone_sightline(mu[q], S[q], ns, None, burn=burn, momenta=mom[q])
                    for q in range(nsl)])
    np.testing.assert_allclose(out_w, ref, rtol=0, atol=1e-12)


def test_warp_phases_not_positive_definite(host_lib):
    mu = np.zeros((2, 2))
    S = np.array([np.eye(2), [[1.0, 2.0], [2.0, 1.0]]])
    st, out, _ = run(host_lib, mu, S, np.ones((2, 3, 2)), 1, warp=True)
    assert st == 1 and np.all(np.isnan(out[1])) and np.all(np.isfinite(out[0]))
