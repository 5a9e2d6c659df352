// Exact Hamiltonian Monte Carlo for one sightline's Gaussian predictive
// truncated to a non-decreasing sequence of log-extinctions (Sect. 5,
// conditioning on dA/ds >= 0).  The sampler is the exact HMC of Pakman &
// Paninski (2014, "Exact Hamiltonian Monte Carlo for truncated multivariate
// Gaussians"), written here in the coordinates y = x - mu instead of the
// whitened z = L^-1 (x - mu):
//
//   * a step draws p ~ N(0, I) and sets the velocity w = L p (S = L L^T);
//   * the motion is y(t) = y cos t + w sin t, w(t) = -y sin t + w cos t, for
//     a total time pi / 2;
//   * wall j is (mu + y)_{j+1} - (mu + y)_j = 0.  With a = y_{j+1} - y_j,
//     b = w_{j+1} - w_j and c = mu_{j+1} - mu_j the difference along the
//     motion is c + r cos(t - phi), r = hypot(a, b), phi = atan2(b, a); when
//     r > |c| it reaches zero at t = phi +- acos(-c / r);
//   * at the first outward hit the velocity is mirrored in the wall.  In z
//     that is v -= 2 (n.v / n.n) n for the wall normal n = L^T f_j
//     (f_j = e_{j+1} - e_j); in y it reads w -= 2 (b / f_j^T S f_j) S f_j.
//
// Every routine takes strided views: element i of a per-sightline vector is
// at p[i * st] and element (a, b) of an m x m matrix at p[(a * m + b) * st],
// so that one thread per sightline with st = number of sightlines reads
// consecutive addresses across a warp.  The routines compile for the device
// (the sampler kernel) and for the host (a check of the same arithmetic
// without a GPU).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define GM_HD __host__ __device__
#else
#define GM_HD
#endif

namespace gmhmc {

constexpr int kMaxWallHits = 10000;  // wall hits within one step, then the step ends
constexpr double kHitEps = 1e-12;    // earlier "hits" are the wall just left
constexpr double kHalfPi = 1.57079632679489661923;
constexpr double kTwoPi = 6.28318530717958647692;

enum : unsigned { kNotPD = 1u, kHitLimit = 2u };

// Covariance entry (a, b) read from the lower triangle.
GM_HD inline double sym(const double* S, int m, int64_t st, int a, int b) {
  return a >= b ? S[(int64_t)(a * m + b) * st] : S[(int64_t)(b * m + a) * st];
}

// Lower Cholesky factor L of S (lower triangle of both); false when S is not
// positive definite.
GM_HD inline bool cholesky(const double* S, double* L, int m, int64_t st) {
  for (int j = 0; j < m; ++j) {
    double d = S[(int64_t)(j * m + j) * st];
    for (int k = 0; k < j; ++k) {
      const double v = L[(int64_t)(j * m + k) * st];
      d -= v * v;
    }
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    L[(int64_t)(j * m + j) * st] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = S[(int64_t)(i * m + j) * st];
      for (int k = 0; k < j; ++k)
        v -= L[(int64_t)(i * m + k) * st] * L[(int64_t)(j * m + k) * st];
      L[(int64_t)(i * m + j) * st] = v / d;
    }
  }
  return true;
}

// First outward wall hit in (kHitEps, t_left]: the wall's index (-1: none)
// and its time in *t_hit.  Ties keep the lower wall index.
GM_HD inline int first_hit(const double* mu, const double* y, const double* w, int m,
                           int64_t st, double t_left, double* t_hit) {
  int best = -1;
  double bt = 0.0;
  for (int j = 0; j + 1 < m; ++j) {
    const double a = y[(int64_t)(j + 1) * st] - y[(int64_t)j * st];
    const double b = w[(int64_t)(j + 1) * st] - w[(int64_t)j * st];
    const double c = mu[(int64_t)(j + 1) * st] - mu[(int64_t)j * st];
    const double r = hypot(a, b);
    if (r <= fabs(c)) continue;  // the motion never reaches this wall
    const double ph = atan2(b, a);
    const double ac = acos(-c / r);
    for (int s = 0; s < 2; ++s) {
      double t = fmod(s == 0 ? ph + ac : ph - ac, kTwoPi);
      if (t < 0.0) t += kTwoPi;
      if (t > kHitEps && t <= t_left) {
        const double deriv = -a * sin(t) + b * cos(t);  // outward: decreasing
        if (deriv < 0.0 && (best < 0 || t < bt)) {
          best = j;
          bt = t;
        }
      }
    }
  }
  *t_hit = bt;
  return best;
}

GM_HD inline void rotate(double* y, double* w, int m, int64_t st, double t) {
  const double ct = cos(t), sn = sin(t);
  for (int i = 0; i < m; ++i) {
    const double yi = y[(int64_t)i * st], wi = w[(int64_t)i * st];
    y[(int64_t)i * st] = yi * ct + wi * sn;
    w[(int64_t)i * st] = -yi * sn + wi * ct;
  }
}

// Mirror the velocity in wall j (see the header comment).
GM_HD inline void reflect(const double* S, double* w, int m, int64_t st, int j) {
  const double b = w[(int64_t)(j + 1) * st] - w[(int64_t)j * st];
  const double nn = sym(S, m, st, j + 1, j + 1) + sym(S, m, st, j, j) -
                    2.0 * sym(S, m, st, j + 1, j);
  const double f = 2.0 * b / nn;
  for (int i = 0; i < m; ++i)
    w[(int64_t)i * st] -= f * (sym(S, m, st, i, j + 1) - sym(S, m, st, i, j));
}

// n_burn + n_samples exact-HMC steps for one sightline.
//   mu, S: the predictive (strided); L, y, w: scratch (strided, m x m, m, m);
//   p: the steps' standard normal momenta, (n_burn + n_samples) x m, contiguous;
//   out: n_samples x m samples of x = mu + y, contiguous;
//   *hits: wall hits over all steps.
// The chain starts from x0 = running maximum of mu, point i raised by 1e-9 i.
// Returns kNotPD (samples NaN) or kHitLimit (a step ended at the wall-hit
// limit before its time was used), else 0.
GM_HD inline unsigned sample_sightline(const double* mu, const double* S, double* L, double* y,
                                       double* w, int64_t st, const double* p, double* out,
                                       int m, int n_burn, int n_samples, int64_t* hits) {
  *hits = 0;
  if (!cholesky(S, L, m, st)) {
    for (int64_t k = 0; k < (int64_t)n_samples * m; ++k) out[k] = NAN;
    return kNotPD;
  }
  double run = 0.0;
  for (int i = 0; i < m; ++i) {
    const double mi = mu[(int64_t)i * st];
    run = (i == 0 || mi > run) ? mi : run;
    y[(int64_t)i * st] = (run + 1e-9 * i) - mi;
  }
  unsigned status = 0;
  int64_t n_hits = 0;
  for (int it = 0; it < n_burn + n_samples; ++it) {
    const double* pk = p + (int64_t)it * m;
    for (int i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int k = 0; k <= i; ++k) acc += L[(int64_t)(i * m + k) * st] * pk[k];
      w[(int64_t)i * st] = acc;
    }
    double t_left = kHalfPi;
    int n = 0;
    for (; n < kMaxWallHits; ++n) {
      double th;
      const int j = first_hit(mu, y, w, m, st, t_left, &th);
      if (j < 0) {
        rotate(y, w, m, st, t_left);
        break;
      }
      rotate(y, w, m, st, th);
      reflect(S, w, m, st, j);
      t_left -= th;
      ++n_hits;
    }
    if (n == kMaxWallHits) status |= kHitLimit;
    if (it >= n_burn) {
      double* o = out + (int64_t)(it - n_burn) * m;
      for (int i = 0; i < m; ++i) o[i] = mu[(int64_t)i * st] + y[(int64_t)i * st];
    }
  }
  *hits = n_hits;
  return status;
}

}  // namespace gmhmc

// ---------------------------------------------------------------------------
// The same chain with one warp per sightline (m <= 32): lane i holds point i.
// A step is a sequence of phases; between phases the lanes synchronise (a
// warp barrier on the device, lane after lane on the host), and every value a
// lane reads from another lane goes through the per-warp arrays of WarpState.
// The arithmetic of each value is the one of sample_sightline (same formulas,
// same order of the sums), so both give the same chain.
namespace gmhmc {

constexpr int kWarpMax = 32;

struct WarpState {
  double* S;   // m x m, both triangles (from the lower one)
  double* L;   // m x m, lower
  double y[kWarpMax], w[kWarpMax], p[kWarpMax], t[kWarpMax];
  double mu[kWarpMax];
  double t_left, fref;
  int64_t nhits;
  unsigned status;
  int pad;
};

// Staging by lane i: mu_i, row i of S (from the lower triangle), the start.
GM_HD inline void w_stage(WarpState& W, int i, int m, const double* mu, const double* S,
                          int64_t st) {
  if (i >= m) return;
  W.mu[i] = mu[(int64_t)i * st];
  for (int k = 0; k < m; ++k) W.S[i * m + k] = sym(S, m, st, i, k);
}

// Lane 0: Cholesky factor, start, counters (after w_stage).
GM_HD inline void w_setup(WarpState& W, int m) {
  W.status = cholesky(W.S, W.L, m, 1) ? 0u : (unsigned)kNotPD;
  double run = 0.0;
  for (int i = 0; i < m; ++i) {
    const double mi = W.mu[i];
    run = (i == 0 || mi > run) ? mi : run;
    W.y[i] = (run + 1e-9 * i) - mi;
  }
  W.nhits = 0;
}

// Lane i: its momentum, then (next phase) its velocity w_i = sum_k L_ik p_k.
GM_HD inline void w_momentum(WarpState& W, int i, int m, const double* pk) {
  if (i < m) W.p[i] = pk[i];
}
GM_HD inline void w_velocity(WarpState& W, int i, int m) {
  if (i >= m) return;
  double acc = 0.0;
  for (int k = 0; k <= i; ++k) acc += W.L[i * m + k] * W.p[k];
  W.w[i] = acc;
}

// Lane j < m - 1: the first outward hit of wall j within t_left (or -1).
GM_HD inline void w_hit(WarpState& W, int j, int m) {
  if (j + 1 >= m) return;
  W.t[j] = -1.0;
  const double a = W.y[j + 1] - W.y[j];
  const double b = W.w[j + 1] - W.w[j];
  const double c = W.mu[j + 1] - W.mu[j];
  const double r = hypot(a, b);
  if (r <= fabs(c)) return;
  const double ph = atan2(b, a);
  const double ac = acos(-c / r);
  double bt = -1.0;
  for (int s = 0; s < 2; ++s) {
    double t = fmod(s == 0 ? ph + ac : ph - ac, kTwoPi);
    if (t < 0.0) t += kTwoPi;
    if (t > kHitEps && t <= W.t_left) {
      const double deriv = -a * sin(t) + b * cos(t);
      if (deriv < 0.0 && (bt < 0.0 || t < bt)) bt = t;
    }
  }
  W.t[j] = bt;
}

// Any lane (all compute the same): the earliest wall, lowest index on ties.
GM_HD inline int w_best(const WarpState& W, int m, double* tb) {
  int best = -1;
  double bt = 0.0;
  for (int j = 0; j + 1 < m; ++j)
    if (W.t[j] >= 0.0 && (best < 0 || W.t[j] < bt)) {
      best = j;
      bt = W.t[j];
    }
  *tb = bt;
  return best;
}

// Lane i: rotate its own (y_i, w_i) by t.
GM_HD inline void w_rotate(WarpState& W, int i, int m, double t) {
  if (i >= m) return;
  const double ct = cos(t), sn = sin(t);
  const double yi = W.y[i], wi = W.w[i];
  W.y[i] = yi * ct + wi * sn;
  W.w[i] = -yi * sn + wi * ct;
}

// Lane 0: the reflection factor of wall j from the rotated velocity.
GM_HD inline void w_reflect_factor(WarpState& W, int m, int j) {
  const double b = W.w[j + 1] - W.w[j];
  const double nn = W.S[(j + 1) * m + j + 1] + W.S[j * m + j] - 2.0 * W.S[(j + 1) * m + j];
  W.fref = 2.0 * b / nn;
}

// Lane i: mirror its velocity component in wall j.
GM_HD inline void w_reflect(WarpState& W, int i, int m, int j) {
  if (i >= m) return;
  W.w[i] -= W.fref * (W.S[i * m + j + 1] - W.S[i * m + j]);
}

}  // namespace gmhmc
