// Quadrature rules computed on the host at context creation.
//
// Gauss-Legendre: the n roots of P_n, refined by Newton's method on the
// Legendre three-term recurrence from the leading-order asymptotic guess
// cos(pi (k + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
//
// Gauss-Hermite (weight exp(-x^2)): roots of the orthonormal Hermite
// polynomial h_n, located by a sign-change scan over the oscillatory region
// |x| < sqrt(2n+1) + 1 and polished by Newton's method (h_n' = sqrt(2n) h_{n-1});
// weights 2 / h_n'(x)^2, returned multiplied by exp(x^2) so that
// int f(x) dx ~ sum w_k exp(x_k^2) f(x_k).
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

static void legendre_eval(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double z = std::cos(pi * (k + 0.75) / (n + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_eval(n, z, &p, &dp);
    // roots come out in decreasing order; store ascending
    x[n - 1 - k] = z;
    w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static double hermite_orthonormal(int n, double x, double* hm1) {
  // h_0 = pi^(-1/4); h_{k+1} = sqrt(2/(k+1)) x h_k - sqrt(k/(k+1)) h_{k-1}
  const double pi = 3.14159265358979323846;
  double h0 = std::pow(pi, -0.25), h1 = std::sqrt(2.0) * x * h0;
  if (n == 0) {
    *hm1 = 0;
    return h0;
  }
  for (int k = 1; k < n; ++k) {
    double h2 = std::sqrt(2.0 / (k + 1.0)) * x * h1 - std::sqrt((double)k / (k + 1.0)) * h0;
    h0 = h1;
    h1 = h2;
  }
  *hm1 = h0;
  return h1;
}

void gauss_hermite(int n, double* x, double* wx) {
  const double lim = std::sqrt(2.0 * n + 1.0) + 1.0;
  const double step = 1e-3;
  std::vector<double> roots;
  double hm1;
  double xa = -lim, fa = hermite_orthonormal(n, xa, &hm1);
  for (double xb = -lim + step; xb <= lim + step && (int)roots.size() < n; xb += step) {
    double fb = hermite_orthonormal(n, xb, &hm1);
    if ((fa < 0) != (fb < 0)) {
      // bisection to a tight bracket, then Newton
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi), fm = hermite_orthonormal(n, mid, &hm1);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      double z = 0.5 * (lo + hi);
      for (int it = 0; it < 5; ++it) {
        double h = hermite_orthonormal(n, z, &hm1);
        double dh = std::sqrt(2.0 * n) * hm1;
        z -= h / dh;
      }
      roots.push_back(z);
    }
    xa = xb;
    fa = fb;
  }
  for (int k = 0; k < n; ++k) {
    double z = k < (int)roots.size() ? roots[k] : 0.0;
    hermite_orthonormal(n, z, &hm1);
    double dh = std::sqrt(2.0 * n) * hm1;
    x[k] = z;
    wx[k] = 2.0 / (dh * dh) * std::exp(z * z);
  }
}

}  // namespace gm
