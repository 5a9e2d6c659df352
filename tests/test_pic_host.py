"""The dense steps of the device PIC posterior (csrc/gm_dense.cuh: Cholesky
in barrier-separated phases, solves, the per-output sums) compiled for the
host and run in the device's launch order — the factorisation phases with
several emulated threads per matrix — on covariance blocks from the oracle,
against the oracle's direct PITC conditioning and its block-site EP
(oracle/pic.py).  CPU only; the device run is checked on a GPU."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import pic as P
from synth import catalogue_subset, make_catalogue

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1708_09705_gb300", "csrc")

HARNESS = r"""
#include "gm_dense.cuh"
#include <vector>
#include <cstring>
using namespace gmdense;
// one factorisation as the device runs it: nt threads, barrier after each phase
static bool chol(double* A, int n, int nt) {
  for (int j = 0; j < n; ++j) {
    const double d = chol_diag(A, n, j);
    if (!(d > 0.0)) return false;
    for (int t = 0; t < nt; ++t) chol_col(A, n, n, j, d, t, nt);
    for (int t = 0; t < nt; ++t) chol_update(A, n, n, j, t, nt);
  }
  return true;
}
extern "C" int pic_host(long n, int R, int nb, const long* boff, const double* Kkk,
                        const double* Kku, const double* Kuu, const double* mu_u,
                        const double* atil, const double* m, const double* sig2, int nt,
                        double* mean, double* cov) {
  const long RR = (long)R * R;
  std::vector<double> Lu(Kuu, Kuu + RR), A(n * R), X, yv(n), Lam(RR), eta(R), Kinv(RR), Pm(RR),
      h(R);
  if (!chol(Lu.data(), R, nt)) return 1;
  for (long j = 0; j < n; ++j) a_row(Lu.data(), R, Kku + j * R, A.data() + j * R);
  std::vector<long> coff(nb + 1, 0);
  for (int k = 0; k < nb; ++k) coff[k + 1] = coff[k] + (boff[k + 1] - boff[k]) * (boff[k + 1] - boff[k]);
  std::vector<double> Cm(coff[nb]);
  for (int k = 0; k < nb; ++k) {
    const long N = boff[k + 1] - boff[k];
    for (long a = 0; a < N; ++a)
      for (long b = 0; b <= a; ++b) {
        const long ra = boff[k] + a, rb = boff[k] + b;
        Cm[coff[k] + a * N + b] = c_entry(Kkk[ra * n + rb], A.data() + ra * R, Kku + rb * R, R,
                                          a == b, sig2[ra]);
      }
    if (N > 0 && !chol(Cm.data() + coff[k], (int)N, nt)) return 2;
  }
  for (long j = 0; j < n; ++j) yv[j] = y_entry(atil[j], m[j], A.data() + j * R, mu_u, R);
  X = A;
  for (int k = 0; k < nb; ++k) {
    const int N = (int)(boff[k + 1] - boff[k]);
    if (N == 0) continue;
    for (int c = 0; c <= R; ++c) {
      if (c < R) solve_lower(Cm.data() + coff[k], N, N, X.data() + boff[k] * R + c, R);
      else solve_lower(Cm.data() + coff[k], N, N, yv.data() + boff[k], 1);
    }
  }
  for (int r1 = 0; r1 < R; ++r1)
    for (int r2 = 0; r2 <= r1; ++r2) Lam[r1 * R + r2] = lambda_entry(X.data(), n, R, r1, r2);
  for (int r = 0; r < R; ++r) eta[r] = eta_entry(X.data(), yv.data(), n, R, r);
  for (int c = 0; c < R; ++c) inverse_col(Lu.data(), R, c, Kinv.data() + c, R);
  for (int r1 = 0; r1 < R; ++r1)
    for (int r2 = 0; r2 <= r1; ++r2) Pm[r1 * R + r2] = Kinv[r1 * R + r2] + Lam[r1 * R + r2];
  for (int r = 0; r < R; ++r) {
    double v = eta[r];
    for (int c = 0; c < R; ++c) v += Kinv[r * R + c] * mu_u[c];
    h[r] = v;
  }
  if (!chol(Pm.data(), R, nt)) return 3;
  for (int r = 0; r < R; ++r) mean[r] = h[r];
  solve_lower(Pm.data(), R, R, mean, 1);
  solve_lower_t(Pm.data(), R, R, mean, 1);
  for (int c = 0; c < R; ++c) inverse_col(Pm.data(), R, c, cov + c, R);
  return 0;
}
"""


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("pic")
    src, so = d / "harness.cpp", d / "libpic_host.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                    f"-I{CSRC}", str(src), "-o", str(so)], check=True)
    L = C.CDLL(str(so))
    vp = C.c_void_p
    L.pic_host.argtypes = [C.c_long, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int,
                           vp, vp]
    L.pic_host.restype = C.c_int
    return L


@pytest.fixture(scope="module")
def setup():
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(150))
    n = len(cat["s"])
    rng = np.random.default_rng(9)
    R = 24
    li = rng.uniform(cat["l"].min(), cat["l"].max(), R)
    bi = rng.uniform(cat["b"].min(), cat["b"].max(), R)
    si = np.exp(rng.uniform(np.log(150), np.log(2500), R))
    union = dict(cat, l=np.concatenate([cat["l"], li]), b=np.concatenate([cat["b"], bi]),
                 s=np.concatenate([cat["s"], si]))
    cv = O.build_cov(union)
    A = np.clip(cat["A_obs"], 0.02, None)
    atil = np.log(A) + 0.02 * rng.standard_normal(n)
    sig2 = (cat["A_sigma"] / A) ** 2
    order = np.argsort(cat["l"])
    groups = [np.sort(g) for g in np.array_split(order, 5)]
    return dict(n=n, R=R, K=cv["K"], m=cv["m"], atil=atil, sig2=sig2, groups=groups,
                u=np.arange(n, n + R))


@pytest.mark.parametrize("nt", [1, 3, 32])
def test_host_pipeline_matches_oracle_pitc(host_lib, setup, nt):
    S = setup
    K, m, u, R = S["K"], S["m"], S["u"], S["R"]
    order = np.concatenate(S["groups"])                # block order of the stars
    boff = np.concatenate([[0], np.cumsum([len(g) for g in S["groups"]])]).astype(np.int64)
    Kkk = np.ascontiguousarray(K[np.ix_(order, order)])
    Kku = np.ascontiguousarray(K[np.ix_(order, u)])
    Kuu = np.ascontiguousarray(K[np.ix_(u, u)])
    mu_u = np.ascontiguousarray(m[u])
    atil = np.ascontiguousarray(S["atil"][order])
    mm = np.ascontiguousarray(m[order])
    sig2 = np.ascontiguousarray(S["sig2"][order])
    mean, cov = np.zeros(R), np.zeros((R, R))
    rc = host_lib.pic_host(len(order), R, len(S["groups"]), boff.ctypes.data, Kkk.ctypes.data,
                           Kku.ctypes.data, Kuu.ctypes.data, mu_u.ctypes.data, atil.ctypes.data,
                           mm.ctypes.data, sig2.ctypes.data, nt, mean.ctypes.data,
                           cov.ctypes.data)
    assert rc == 0
    blocks = [dict(Kku=K[np.ix_(g, u)], Kkk=K[np.ix_(g, g)], m=m[g], atil=S["atil"][g],
                   sig2=S["sig2"][g]) for g in S["groups"]]
    ref_m, ref_c = P.pitc_posterior_direct(Kuu, blocks, mu_u)
    np.testing.assert_allclose(mean, ref_m, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(cov, ref_c, rtol=1e-8, atol=1e-12)
    ep_m, ep_c, _ = P.ep_blocks(Kuu, blocks, mu_u, max_sweeps=2)
    np.testing.assert_allclose(mean, ep_m, rtol=1e-8, atol=1e-10)


def test_host_cholesky_phases_detect_indefinite(host_lib, setup):
    S = setup
    R = S["R"]
    Kuu = -np.eye(R)
    z = np.zeros(1)
    one = np.array([0, 1], dtype=np.int64)
    rc = host_lib.pic_host(1, R, 1, one.ctypes.data, np.ones(1).ctypes.data,
                           np.zeros(R).ctypes.data, Kuu.ctypes.data, np.zeros(R).ctypes.data,
                           z.ctypes.data, z.ctypes.data, np.ones(1).ctypes.data, 2,
                           np.zeros(R).ctypes.data, np.zeros((R, R)).ctypes.data)
    assert rc == 1
