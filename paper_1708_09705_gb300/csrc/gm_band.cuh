// Band rule for the sightline double integral of the covariance (Sect. 3):
//
//   R_ij = I_ij / (s_i s_j),
//   I_ij = int_0^si int_0^sj g(|t u_i - t' u_j|) dt' dt,
//
// integrated in the coordinates d = t - t', m = (t + t') / 2 (unit
// Jacobian), where |t u_i - t' u_j|^2 = d^2 (1 - c^2/4) + m^2 c^2 with
// c^2 = |u_i - u_j|^2 and, for each d, m runs over
// [|d|/2, min(si - d/2, sj + d/2)].  Lengths are in units of the outer
// scale L0 (the rule is scale-free), and g is a function of x = r^2 / L0^2.
//
//   * d: breakpoints 0, +-h0, +-h0 (1 + q), +-h0 (1 + q + q^2), ... clipped at
//     min(si, K) on the positive side and min(sj, K) on the negative side
//     (geometric grading towards the cusp of g at r = 0), plus the kink
//     d = si - sj of the inner interval; n-point Gauss-Legendre per panel.
//   * m, for c > 0: breakpoints from the lower end with widths
//     m0 (1/c) q^k, up to the upper end or K / c beyond the lower end (the
//     integrand decays on the scale L0 / c); n-point Gauss-Legendre per
//     panel.  For c = 0 the inner integrand does not depend on m and the
//     inner integral is (upper - lower) g(d^2).
//
// The routines compile for the device (the band-rule quadrature kernels,
// one warp per pair with the lanes over the d-nodes) and for the host (a
// check of the node set and the sums without a GPU).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define GM_HD __host__ __device__
#else
#define GM_HD
#endif

namespace gmband {

constexpr int kN = 6;          // Gauss-Legendre nodes per panel
constexpr double kH0 = 1e-3;   // first d-panel width (units of L0)
constexpr double kQ = 3.0;     // panel growth ratio
constexpr double kM0 = 0.25;   // first m-panel width (units of L0 / c)
constexpr double kK = 40.0;    // truncation (units of L0): g(40 L0) < 2e-18 sigma2

// Gauss-Legendre nodes and weights of [0, 1], n = 6: (1 + x_i) / 2 for the
// roots x_i of P_6, ascending, and half the weights.
GM_HD inline double gl_z(int i) {
  switch (i) {
    case 0: return 0.03376524289842403;
    case 1: return 0.16939530676686776;
    case 2: return 0.38069040695840156;
    case 3: return 0.6193095930415985;
    case 4: return 0.8306046932331322;
    default: return 0.9662347571015759;
  }
}
GM_HD inline double gl_w(int i) {
  switch (i) {
    case 0: case 5: return 0.08566224618958514;
    case 1: case 4: return 0.18038078652406936;
    default: return 0.23395696728634552;
  }
}

// Number of panels of one side [0, D] (D > 0): the smallest k with
// h0 (q^k - 1) / (q - 1) >= D.
GM_HD inline int side_panels(double D) {
  if (!(D > 0.0)) return 0;
  int k = (int)ceil(log1p(D * (kQ - 1.0) / kH0) / log(kQ));
  if (k < 1) k = 1;
  // guard the rounding of the logarithm: the last breakpoint must reach D
  while (kH0 * (pow(kQ, (double)k) - 1.0) / (kQ - 1.0) < D) ++k;
  while (k > 1 && kH0 * (pow(kQ, (double)(k - 1)) - 1.0) / (kQ - 1.0) >= D) --k;
  return k;
}

// Breakpoint j (0..np) of one side, clipped at D.
GM_HD inline double side_point(int j, int np, double D) {
  if (j >= np) return D;
  const double v = kH0 * (pow(kQ, (double)j) - 1.0) / (kQ - 1.0);
  return v < D ? v : D;
}

// The merged d-breakpoints of one pair: negative side, 0, positive side, and
// the kink si - sj when it falls strictly inside a panel.
struct Geometry {
  double A, B, c2;  // si / L0, sj / L0, chord^2
  double Dp, Dn;    // extent of the positive and negative sides
  int np, nn;       // panels on each side
  double kink;
  int kidx;         // index the kink takes in the merged list (-1: not inserted)
  int npanels;      // panels of the merged list

  GM_HD double base(int i) const {  // i in [0, nn + np]
    return i < nn ? -side_point(nn - i, nn, Dn) : side_point(i - nn, np, Dp);
  }
  GM_HD double point(int i) const {
    if (kidx < 0 || i < kidx) return base(i);
    return i == kidx ? kink : base(i - 1);
  }
};

GM_HD inline Geometry geometry(double A, double B, double c2) {
  Geometry g;
  g.A = A;
  g.B = B;
  g.c2 = c2;
  g.Dp = A < kK ? A : kK;
  g.Dn = B < kK ? B : kK;
  g.np = side_panels(g.Dp);
  g.nn = side_panels(g.Dn);
  g.kink = A - B;
  g.kidx = -1;
  const int nbase = g.nn + g.np + 1;
  if (g.kink > -g.Dn && g.kink < g.Dp) {
    // first base point >= kink (the base list is sorted)
    int lo = 0, hi = nbase - 1;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (g.base(mid) < g.kink) lo = mid + 1; else hi = mid;
    }
    if (g.base(lo) != g.kink) g.kidx = lo;
  }
  g.npanels = nbase - 1 + (g.kidx >= 0 ? 1 : 0);
  return g;
}

// Contribution of d-node k (panel k / kN, node k % kN) of the pair:
// w_d * int g dm.  G: callable g(x) with x = r^2 / L0^2 in the arithmetic
// type T of the inner sum (the panel geometry is always double).
template <typename T, typename G>
GM_HD inline T d_node(const Geometry& geo, int k, const G& gfun) {
  const int p = k / kN, i = k - p * kN;
  const double a = geo.point(p), b = geo.point(p + 1);
  const double dk = a + (b - a) * gl_z(i);
  const double wk = (b - a) * gl_w(i);
  const double lo = fabs(dk) * 0.5;
  const double u1 = geo.A - dk * 0.5, u2 = geo.B + dk * 0.5;
  const double hi = u1 < u2 ? u1 : u2;
  if (!(hi > lo) || wk == 0.0) return (T)0;
  if (geo.c2 == 0.0) return (T)(wk * (hi - lo)) * gfun((T)(dk * dk));
  const double c = sqrt(geo.c2);
  const double sc = 1.0 / c;
  const T dd = (T)(dk * dk * (1.0 - 0.25 * geo.c2));
  const T c2 = (T)geo.c2;
  const double lim = lo + kK * sc;
  const double end = hi < lim ? hi : lim;
  T acc = 0;
  double ma = lo, h = kM0 * sc;
  while (ma < end) {
    const double mb = ma + h < end ? ma + h : end;
    const T m0 = (T)ma, len = (T)(mb - ma);
    T s = 0;
    for (int j = 0; j < kN; ++j) {
      const T m = m0 + len * (T)gl_z(j);
      s += (T)gl_w(j) * gfun(dd + m * m * c2);
    }
    acc += len * s;
    ma = mb;
    h *= kQ;
  }
  return (T)wk * acc;
}

GM_HD inline int d_nodes(const Geometry& geo) { return geo.npanels * kN; }

}  // namespace gmband
