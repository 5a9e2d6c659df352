"""The band-rule routines of the device quadrature (csrc/gm_band.cuh)
compiled for the host, with the exact kernel g, against the oracle's band
rule (oracle/band.py) with the same parameters: the same node set (number of
integrand evaluations) and the same integral.  CPU only; the device kernels
that use these routines are checked against the oracle on a GPU."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import band as Bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1708_09705_gb300", "csrc")
RULE = dict(n=6, h0=1e-3, q=3.0, m0=0.25, K=40.0)   # the device rule's constants

# g(x) = expm1(sigma2 phi(sqrt(x))) (lognormal form), phi the von Karman
# correlation of order 1/3, x = r^2 / L0^2.
HARNESS = r"""
#include "gm_band.cuh"
#include <cmath>
struct Gexact {
  double sigma2; long* count;
  double operator()(double x) const {
    ++*count;
    const double y = std::sqrt(x);
    const double nu = 1.0 / 3.0;
    const double phi = y > 0 ? std::pow(2.0, 1.0 - nu) / std::tgamma(nu) * std::pow(y, nu) *
                                   std::cyl_bessel_k(nu, y)
                             : 1.0;
    return std::expm1(sigma2 * phi);
  }
};
extern "C" double band_R_host(double A, double B, double c2, double sigma2, long* evals) {
  gmband::Geometry geo = gmband::geometry(A, B, c2);
  Gexact g{sigma2, evals};
  *evals = 0;
  double acc = 0.0;
  for (int k = 0; k < gmband::d_nodes(geo); ++k) acc += gmband::d_node<double>(geo, k, g);
  return acc / (A * B);
}
extern "C" int band_panels_host(double A, double B, double c2, double* pts, int cap) {
  gmband::Geometry geo = gmband::geometry(A, B, c2);
  for (int i = 0; i <= geo.npanels && i < cap; ++i) pts[i] = geo.point(i);
  return geo.npanels;
}
"""


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("band")
    src, so = d / "harness.cpp", d / "libband_host.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                    f"-I{CSRC}", str(src), "-o", str(so)], check=True)
    L = C.CDLL(str(so))
    L.band_R_host.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                              C.POINTER(C.c_long)]
    L.band_R_host.restype = C.c_double
    L.band_panels_host.argtypes = [C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_int]
    L.band_panels_host.restype = C.c_int
    return L


PAIRS = [(40.0, 40.0, 0.0), (100.0, 130.0, 0.0), (3000.0, 2950.0, 0.0), (100.0, 120.0, 0.04),
         (1000.0, 1020.0, 1e-4), (3000.0, 2990.0, 2.5e-5), (150.0, 180.0, 0.04),
         (500.0, 480.0, 0.0064), (25.0, 700.0, 1e-3), (2000.0, 2000.0, 1e-6)]


@pytest.mark.parametrize("si,sj,c2", PAIRS)
def test_host_build_matches_oracle_band_rule(host_lib, si, sj, c2):
    L0, sigma2 = 20.0, 1.0
    ev = C.c_long(0)
    got = host_lib.band_R_host(si / L0, sj / L0, c2, sigma2, C.byref(ev))
    ref, evr = Bd.pair_R_band(si, sj, c2, lambda r: O.g_of_r(r, sigma2, L0), L0, **RULE)
    # the same node set, up to panels of rounding width where a panel end
    # and the end of the interval coincide mathematically (counted on one
    # side, not the other; they carry no weight)
    assert abs(ev.value - evr[0]) <= 0.02 * evr[0]
    assert got == pytest.approx(ref[0], rel=1e-12)


def test_breakpoints_are_the_oracle_set(host_lib):
    L0 = 20.0
    for si, sj, c2 in PAIRS:
        pts = np.zeros(128)
        npn = host_lib.band_panels_host(si / L0, sj / L0, c2, pts.ctypes.data, 128)
        d, _, _ = Bd.band_nodes(si, sj, c2, L0, **RULE)
        # the oracle's d-nodes are the device's panels mapped to pc
        z = 0.5 * (1 + np.polynomial.legendre.leggauss(6)[0])
        a, b = pts[:npn] * L0, pts[1:npn + 1] * L0
        dev_nodes = (a[:, None] + (b - a)[:, None] * z[None, :]).ravel()
        np.testing.assert_allclose(np.unique(d), np.unique(dev_nodes[(b - a).repeat(6) > 0]),
                                   rtol=1e-13, atol=1e-12)
