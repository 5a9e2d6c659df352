"""Pins of the band rule for the sightline double integral (oracle/band.py):
nested adaptive quadrature in the original (t, t') coordinates, exactness on
polynomial and constant kernels, and the size of the literal Gauss-Legendre
rule's error that it removes.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from oracle import band as Bd

L0 = 20.0


def g(r):
    return O.g_of_r(r, 1.0, L0)


def nested_adaptive(si, sj, c2):
    """I / (si sj) by nested scipy quad over t' (inner, with the ridge t' = t
    as a breakpoint) and t (outer), in the original coordinates."""
    def inner(t):
        f = lambda tp: float(g(np.array([math.sqrt((t - tp) ** 2 + t * tp * c2)]))[0])  # noqa: E731
        pts = [p for p in (t - 5 * L0, t - L0, t, t + L0, t + 5 * L0) if 0 < p < sj]
        return integrate.quad(f, 0.0, sj, points=pts or None, epsabs=0, epsrel=1e-12,
                              limit=400)[0]
    pts = [p for p in (L0, 5 * L0, sj - 5 * L0, sj, sj + 5 * L0) if 0 < p < si]
    v = integrate.quad(inner, 0.0, si, points=sorted(set(pts)) or None, epsabs=0,
                       epsrel=1e-10, limit=400)[0]
    return v / (si * sj)


@pytest.mark.parametrize("si,sj", [(40.0, 40.0), (100.0, 130.0), (1000.0, 1000.0),
                                   (3000.0, 2950.0)])
def test_same_direction_against_nested_adaptive(si, sj):
    R, _ = Bd.pair_R_band(si, sj, 0.0, g, L0)
    assert R[0] == pytest.approx(nested_adaptive(si, sj, 0.0), rel=2e-8)


@pytest.mark.parametrize("si,sj,c", [(100.0, 120.0, 0.2), (1000.0, 1020.0, 0.01),
                                     (3000.0, 2990.0, 0.005), (500.0, 480.0, 0.08)])
def test_diverging_sightlines_against_nested_adaptive(si, sj, c):
    R, _ = Bd.pair_R_band(si, sj, c * c, g, L0)
    assert R[0] == pytest.approx(nested_adaptive(si, sj, c * c), rel=1e-6)


def test_polynomial_and_constant_kernels_are_exact():
    """Without truncation the rule is piecewise Gauss-Legendre over panels
    whose ends include every kink of the domain, so r^2 and r^4 (polynomials
    of degree 2 and 4 in (d, m)) and constants come out exactly."""
    rng = np.random.default_rng(1)
    si, sj = rng.uniform(50, 3000, 8), rng.uniform(50, 3000, 8)
    ct = np.cos(rng.uniform(0, 0.2, 8))
    c2 = 2 - 2 * ct
    nt = dict(K=1e12, n=4)
    R2, _ = Bd.pair_R_band(si, sj, c2, lambda r: r ** 2, L0, **nt)
    np.testing.assert_allclose(R2, (si ** 2 + sj ** 2) / 3.0 - ct * si * sj / 2.0, rtol=1e-12)
    R4, _ = Bd.pair_R_band(si, sj, c2, lambda r: r ** 4, L0, **nt)
    ref4 = (si ** 4 / 5 + sj ** 4 / 5 + 4 * ct * ct * si ** 2 * sj ** 2 / 9
            + 2 * si ** 2 * sj ** 2 / 9 - ct * si ** 3 * sj / 2 - ct * si * sj ** 3 / 2)
    np.testing.assert_allclose(R4, ref4, rtol=1e-11)
    R0, _ = Bd.pair_R_band(si, sj, c2, lambda r: np.full_like(r, 0.7), L0, **nt)
    np.testing.assert_allclose(R0, 0.7, rtol=1e-13)


def test_literal_rule_error_that_the_band_rule_removes():
    """The diagonal at 3000 pc (outer scale 20 pc): the 64-node Gauss-Legendre
    rule of the covariance assembly is off by more than 100 %; the band rule
    agrees with the one-dimensional reduction 2/s^2 int_0^s (s - r) g(r) dr."""
    s = 3000.0
    ex = 2 / s ** 2 * integrate.quad(lambda r: (s - r) * g(r), 0, s, epsabs=0, epsrel=1e-13,
                                     limit=2000, points=[1e-6, 1e-3, 1e-1, 1, 10, 100])[0]
    gl64 = O.pair_R(np.array([s]), np.array([s]), np.zeros(1), g, 64)[0]
    band, ev = Bd.pair_R_band(s, s, 0.0, g, L0)
    assert gl64 / ex - 1 > 1.0
    assert band[0] == pytest.approx(ex, rel=1e-8)
    assert ev[0] < 4096
