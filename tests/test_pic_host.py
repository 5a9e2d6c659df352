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
// the whole device pipeline after the quadrature and neighbour search, in
// its launch order, from the stars' CSR and the inducing points' CSR; the
// factors stay in St for the predictive
struct St {
  std::vector<int64_t> boff, coff, bidx;
  std::vector<int32_t> rowpos, dims;
  std::vector<double> Lu, mu_u, Kku, A, C, mean, cov;
};
static int pipeline(St& S, long n, int R, int nb, const int32_t* blk, const int64_t* row_ptr,
                    const int32_t* col, const double* val, const int64_t* qptr,
                    const int32_t* qcol, const double* qval, long qnnz, const double* us,
                    const double* ux, const double* uy, const double* uz, const double* kp,
                    double inv_cut, int taper, int form, double log_rho_bar, double sigma2,
                    const double* obs, const double* sig, const double* prior_m, int nt,
                    double* si, double* sj, double* ch) {
  S.boff.resize(nb + 1); S.coff.resize(nb + 1); S.bidx.resize(n); S.rowpos.resize(n);
  S.dims.resize(nb);
  if (!gmpic::block_lists(n, blk, nb, 8192, S.boff.data(), S.coff.data(), S.bidx.data(),
                          S.rowpos.data(), S.dims.data()))
    return 9;
  const long RR = (long)R * R, np = (long)R * (R + 1) / 2;
  std::vector<double> Kuu(RR, 0.0), X, yv(n), Lam(RR), eta(R), Kinv(RR), Pm(RR), h(R);
  S.mu_u.assign(R, 0.0); S.Kku.assign(n * R, 0.0); S.A.assign(n * R, 0.0);
  S.C.assign(S.coff[nb], 0.0); S.mean.assign(R, 0.0); S.cov.assign(RR, 0.0);
  for (long e = 0; e < qnnz; ++e) gmpic::kku_entry(e, R, qptr, qcol, qval, S.rowpos.data(), S.Kku.data());
  for (long p = 0; p < np; ++p) gmpic::upair(p, us, ux, uy, uz, si, sj, ch);
  for (long p = 0; p < np; ++p)
    gmpic::kuu_entry(p, R, inv_cut, taper, form, log_rho_bar, sigma2, us, ch, kp, Kuu.data(),
                     S.mu_u.data());
  S.Lu = Kuu;
  if (!chol(S.Lu.data(), R, nt)) return 1;
  for (long j = 0; j < n; ++j) a_row(S.Lu.data(), R, S.Kku.data() + j * R, S.A.data() + j * R);
  for (long e = 0; e < S.coff[nb]; ++e)
    gmpic::cmat_entry(e, nb, S.coff.data(), S.boff.data(), R, S.bidx.data(), row_ptr, col, val,
                      S.A.data(), S.Kku.data(), sig, S.C.data());
  for (int k = 0; k < nb; ++k)
    if (S.dims[k] > 0 && !chol(S.C.data() + S.coff[k], S.dims[k], nt)) return 2;
  for (long j = 0; j < n; ++j)
    yv[j] = y_entry(obs[S.bidx[j]], prior_m[S.bidx[j]], S.A.data() + j * R, S.mu_u.data(), R);
  X = S.A;
  for (long t = 0; t < (long)nb * (R + 1); ++t)
    gmpic::fsolve_task(t, R, S.coff.data(), S.boff.data(), S.C.data(), X.data(), yv.data());
  for (long e = 0; e < RR + R; ++e) gmpic::lambda_task(e, n, R, X.data(), yv.data(), Lam.data(), eta.data());
  for (int c = 0; c < R; ++c) inverse_col(S.Lu.data(), R, c, Kinv.data() + c, R);
  for (long e = 0; e < RR + R; ++e)
    gmpic::prec_task(e, R, Kinv.data(), Lam.data(), S.mu_u.data(), eta.data(), Pm.data(), h.data());
  if (!chol(Pm.data(), R, nt)) return 3;
  for (int r = 0; r < R; ++r) S.mean[r] = h[r];
  solve_lower(Pm.data(), R, R, S.mean.data(), 1);
  solve_lower_t(Pm.data(), R, R, S.mean.data(), 1);
  for (int c = 0; c < R; ++c) inverse_col(Pm.data(), R, c, S.cov.data() + c, R);
  return 0;
}

extern "C" int pic_full_host(long n, int R, int nb, const int32_t* blk, const int64_t* row_ptr,
                             const int32_t* col, const double* val, const int64_t* qptr,
                             const int32_t* qcol, const double* qval, long qnnz,
                             const double* us, const double* ux, const double* uy,
                             const double* uz, const double* kp, double inv_cut, int taper,
                             int form, double log_rho_bar, double sigma2, const double* obs,
                             const double* sig, const double* prior_m, int nt, double* mean,
                             double* cov, double* si, double* sj, double* ch,
                             long nq, const int32_t* q_blk, const double* ksu, const double* kss,
                             const double* ms, const int64_t* pptr, const int32_t* pcol,
                             const double* pval, double* pmean, double* pvar) {
  St S;
  const int rc = pipeline(S, n, R, nb, blk, row_ptr, col, val, qptr, qcol, qval, qnnz, us, ux,
                          uy, uz, kp, inv_cut, taper, form, log_rho_bar, sigma2, obs, sig,
                          prior_m, nt, si, sj, ch);
  if (rc) return rc;
  for (int r = 0; r < R; ++r) mean[r] = S.mean[r];
  for (long e = 0; e < (long)R * R; ++e) cov[e] = S.cov[e];
  int maxN = 1;
  for (int k = 0; k < nb; ++k) maxN = S.dims[k] > maxN ? S.dims[k] : maxN;
  std::vector<double> w(3 * R + 2 * maxN);
  for (long q = 0; q < nq; ++q)
    gmpic::pic_point(R, q_blk[q], S.boff.data(), S.coff.data(), S.bidx.data(), S.Lu.data(),
                     S.C.data(), S.A.data(), S.Kku.data(), S.mu_u.data(), S.mean.data(),
                     S.cov.data(), obs, prior_m, ksu + q * R, kss[q], ms[q], pptr[q], pptr[q + 1],
                     pcol, pval, w.data(), w.data() + R, w.data() + 2 * R, w.data() + 3 * R,
                     w.data() + 3 * R + maxN, pmean + q, pvar + q);
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
    L.pic_full_host.argtypes = [C.c_long, C.c_int, C.c_int] + [vp] * 7 + [C.c_long] + [vp] * 5 + \
        [C.c_double, C.c_int, C.c_int, C.c_double, C.c_double] + [vp] * 3 + [C.c_int] + \
        [vp] * 5 + [C.c_long] + [vp] * 9
    L.pic_full_host.restype = C.c_int
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
    # extra query points near stars, assigned to the block of that star
    jq = rng.choice(n, 8, replace=False)
    ql, qb_, qs = cat["l"][jq] + 3e-4, cat["b"][jq] - 3e-4, cat["s"][jq] * 0.93
    union = dict(cat, l=np.concatenate([cat["l"], li, ql]), b=np.concatenate([cat["b"], bi, qb_]),
                 s=np.concatenate([cat["s"], si, qs]))
    cv = O.build_cov(union)
    A = np.clip(cat["A_obs"], 0.02, None)
    atil = np.log(A) + 0.02 * rng.standard_normal(n)
    sig2 = (cat["A_sigma"] / A) ** 2
    order = np.argsort(cat["l"])
    groups = [np.sort(g) for g in np.array_split(order, 5)]
    star_blk = np.zeros(n, dtype=np.int32)
    for k, g in enumerate(groups):
        star_blk[g] = k
    return dict(n=n, R=R, K=cv["K"], m=cv["m"], atil=atil, sig2=sig2, groups=groups,
                u=np.arange(n, n + R), cat=cat, li=li, bi=bi, si=si, ql=ql,
                qblk=star_blk[jq])


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


def test_host_full_pipeline_from_csr_matches_oracle(host_lib, setup):
    """From the stars' CSR, the inducing points' CSR over the stars and the
    inducing pairs' untapered values (the inputs the device gets from its
    quadrature and neighbour search), in the device's launch order."""
    from scipy import sparse
    S = setup
    K, m, u, R, n = S["K"], S["m"], S["u"], S["R"], S["n"]
    cat = S["cat"]
    Ks = sparse.csr_matrix(K[:n, :n])
    Ks.sort_indices()
    Kq = sparse.csr_matrix(K[np.ix_(u, np.arange(n))])
    Kq.sort_indices()
    row_ptr = Ks.indptr.astype(np.int64)
    col = Ks.indices.astype(np.int32)
    val = Ks.data.astype(np.float64)
    qptr = Kq.indptr.astype(np.int64)
    qcol = Kq.indices.astype(np.int32)
    qval = Kq.data.astype(np.float64)
    blk = np.zeros(n, dtype=np.int32)
    for k, g in enumerate(S["groups"]):
        blk[g] = k
    us = S["si"]
    uv = O.unit_vectors(S["li"], S["bi"])
    ux, uy, uz = (np.ascontiguousarray(uv[:, k]) for k in range(3))
    a_idx, b_idx = [], []
    for a in range(R):
        for b in range(a + 1):
            a_idx.append(a)
            b_idx.append(b)
    a_idx, b_idx = np.array(a_idx), np.array(b_idx)
    chord2 = ((uv[a_idx] - uv[b_idx]) ** 2).sum(1)
    L0, sig2 = float(cat["outer_scale_pc"]), float(cat["sigma2"])
    kp = O.K_from_R(O.pair_R(us[a_idx], us[b_idx], chord2,
                             lambda r: O.g_of_r(r, sig2, L0), int(cat["n_nodes"])),
                    O.FORM_LOGNORMAL)
    np_ = len(kp)
    si, sj, ch = np.zeros(np_), np.zeros(np_), np.zeros(np_)
    mean, cov = np.zeros(R), np.zeros((R, R))
    obs = np.ascontiguousarray(S["atil"])
    sig = np.sqrt(S["sig2"])
    pm = np.ascontiguousarray(m[:n])
    # queries: every star (in its block) and the extra points of the fixture
    nqx = len(S["ql"])
    qidx = np.concatenate([np.arange(n), n + R + np.arange(nqx)])
    q_blk = np.concatenate([blk, S["qblk"]]).astype(np.int32)
    ksu = np.ascontiguousarray(K[np.ix_(qidx, u)])
    kss = np.ascontiguousarray(np.diag(K)[qidx])
    ms = np.ascontiguousarray(m[qidx])
    Kp = sparse.csr_matrix(K[np.ix_(qidx, np.arange(n))])
    Kp.sort_indices()
    pptr = Kp.indptr.astype(np.int64)
    pcol = Kp.indices.astype(np.int32)
    pval = Kp.data.astype(np.float64)
    pmean, pvar = np.zeros(len(qidx)), np.zeros(len(qidx))
    rc = host_lib.pic_full_host(
        n, R, len(S["groups"]), blk.ctypes.data, row_ptr.ctypes.data, col.ctypes.data,
        val.ctypes.data, qptr.ctypes.data, qcol.ctypes.data, qval.ctypes.data, len(qval),
        us.ctypes.data, ux.ctypes.data, uy.ctypes.data, uz.ctypes.data, kp.ctypes.data,
        1.0 / float(cat["cutoff_pc"]), 0, 0, np.log(float(cat["rho_bar"])), sig2,
        obs.ctypes.data, sig.ctypes.data, pm.ctypes.data, 4, mean.ctypes.data, cov.ctypes.data,
        si.ctypes.data, sj.ctypes.data, ch.ctypes.data, len(qidx), q_blk.ctypes.data,
        ksu.ctypes.data, kss.ctypes.data, ms.ctypes.data, pptr.ctypes.data, pcol.ctypes.data,
        pval.ctypes.data, pmean.ctypes.data, pvar.ctypes.data)
    assert rc == 0
    np.testing.assert_array_equal(si, us[a_idx])
    np.testing.assert_array_equal(sj, us[b_idx])
    np.testing.assert_allclose(ch * ch, chord2, rtol=1e-12, atol=1e-18)
    blocks = [dict(Kku=K[np.ix_(g, u)], Kkk=K[np.ix_(g, g)], m=m[g], atil=S["atil"][g],
                   sig2=S["sig2"][g]) for g in S["groups"]]
    ref_m, ref_c = P.pitc_posterior_direct(K[np.ix_(u, u)], blocks, m[u])
    np.testing.assert_allclose(mean, ref_m, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(cov, ref_c, rtol=1e-8, atol=1e-12)
    # the PIC predictive at the stars and at the extra points
    Kuu = K[np.ix_(u, u)]
    for q in range(len(qidx)):
        k = q_blk[q]
        g = S["groups"][k]
        b = dict(Kku=K[np.ix_(g, u)], Kkk=K[np.ix_(g, g)], m=m[g], atil=S["atil"][g],
                 sig2=S["sig2"][g])
        j = qidx[q]
        mm_, vv_ = P.pic_predict(Kuu, m[u], ref_m, ref_c, b, K[np.ix_([j], u)], np.diag(K)[[j]],
                                 K[np.ix_([j], g)], m[[j]])
        assert pmean[q] == pytest.approx(mm_[0], rel=1e-9, abs=1e-10)
        assert pvar[q] == pytest.approx(vv_[0], rel=1e-7, abs=1e-12)
