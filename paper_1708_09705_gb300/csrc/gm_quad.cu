// Covariance of log-extinctions by sightline double quadrature (Sect. 3).
//
// For stars i, j at distances s_i, s_j in directions u_i, u_j the density
// covariance is integrated along both sightlines:
//   R_ij = (1 / s_i s_j) int_0^{s_i} int_0^{s_j} g(|t u_i - t' u_j|) dt dt',
// g = expm1(sigma2 phi(r / L0)) (lognormal moment match of rho = exp f) or
// sigma2 phi (first-order form), where phi is the correlation of a
// Kolmogorov spectrum truncated at the outer scale L0 (Sect. 1):
//   phi(x) = 2^(2/3) / Gamma(1/3) x^(1/3) K_(1/3)(x).
// Then K_ij = log1p(R_ij) (or R_ij) times the Wendland taper of the 3-D star
// separation, and m_i = ln(rho_bar s_i) - K_ii / 2.
//
// phi is evaluated once per context on the GPU from the integral
// representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (trapezoid
// rule, exponentially convergent), at the nodes of a log-spaced cubic table
// in x^2 = r^2 / L0^2; each build refits the table of g for the current
// sigma2 and the quadrature kernels interpolate it.  The separation is taken
// in the cancellation-free chord form r^2 = (t - t')^2 + t t' |u_i - u_j|^2.
//
// Two node rules: the Q-node Gauss-Legendre rule on each sightline
// (GM_QUAD_GL), and the band rule of gm_band.cuh (GM_QUAD_BAND), composite
// Gauss-Legendre in d = t - t', m = (t + t')/2 graded towards the cusp of g,
// which converges where s >> L0 (the Q-node rule's nodes are s / Q apart).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gm_band.cuh"
#include "gm_internal.cuh"

namespace gm {

// ------------------------------------------------------------ phi table
__device__ __forceinline__ double seg_lo(const TableGeom g, int k) {
  int oct = k >> g.m, sub = k & ((1 << g.m) - 1);
  return ldexp(1.0 + (double)sub / (double)(1 << g.m), g.emin + oct);
}

// phi(rho) for rho > 0 by the trapezoid rule with step h = 0.1 in t.
__device__ double phi_of_rho(double rho, double cnorm) {
  const double h = 0.1;
  double sum = 0.5 * exp(-rho);  // t = 0 term: exp(-rho) cosh(0)
  for (int k = 1; k < 4000; ++k) {
    double t = k * h;
    double e = exp(t * (1.0 / 3.0));
    double ei = 1.0 / e;
    double ch3 = 0.5 * (e + ei);                 // cosh(t/3)
    double ch = 0.5 * (e * e * e + ei * ei * ei);  // cosh(t)
    double term = exp(-rho * ch) * ch3;
    sum += term;
    // remaining terms are below 1e-20 of the sum once rho (cosh t - 1)
    // exceeds t/3 + 50
    if (rho * (ch - 1.0) > t * (1.0 / 3.0) + 50.0) break;
  }
  return cnorm * cbrt(rho) * (h * sum);
}

__global__ void k_phi_points(TableGeom g, double cnorm, double* __restrict__ out) {
  const int np = g.n_pts();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    int k = p / 3, q = p - 3 * k;
    double x;
    if (k >= g.n_real()) {
      x = ldexp(1.0, g.emax);
    } else {
      double lo = seg_lo(g, k);
      double H = ldexp(1.0 / (double)(1 << g.m), g.emin + (k >> g.m));
      x = lo + H * (double)q / 3.0;
    }
    out[p] = phi_of_rho(sqrt(x), cnorm);
  }
}

// Cubic through g at the four equispaced nodes of each segment (Newton
// forward differences).  FP32 tables hold coefficients of the normalised
// offset v = (x - x_lo) / H in [0, 1) (all O(1)); FP64 tables hold
// coefficients of the absolute offset d = x - x_lo (its range covers 1/H^3).
template <typename T4>
__global__ void k_gtab(TableGeom g, const double* __restrict__ phi, double sigma2, int form,
                       int normalised, T4* __restrict__ tab) {
  const int nr = g.n_real();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= nr; k += gridDim.x * blockDim.x) {
    T4 o;
    if (k == nr) {
      o.x = o.y = o.z = o.w = 0;
    } else {
      double v[4];
      for (int q = 0; q < 4; ++q) {
        double c = sigma2 * phi[3 * k + q];
        v[q] = form == GM_FORM_LOGNORMAL ? expm1(c) : c;
      }
      double d1 = v[1] - v[0], d2 = v[2] - 2 * v[1] + v[0], d3 = v[3] - 3 * v[2] + 3 * v[1] - v[0];
      // p(w) = c0 + c1 w + c2 w^2 + c3 w^3 with w = 3 v
      double c0 = v[0], c1 = d1 - 0.5 * d2 + d3 / 3.0, c2 = 0.5 * d2 - 0.5 * d3, c3 = d3 / 6.0;
      double H = ldexp(1.0 / (double)(1 << g.m), g.emin + (k >> g.m));
      double sc = normalised ? 3.0 : 3.0 / H;
      o.x = c0;
      o.y = c1 * sc;
      o.z = c2 * sc * sc;
      o.w = c3 * sc * sc * sc;
    }
    tab[k] = o;
  }
}

// ------------------------------------------------------------ g lookup
struct TabF32 {
  int base;      // float bits of 2^emin
  int shift;     // 23 - m
  int last;      // index of the zero segment
  float xmin;
};
struct TabF64 {
  int base;      // high word of 2^emin
  int shift;     // 20 - m
  int last;
  double xmin;
};

// v = position of x inside its segment, in [0, 1): the mantissa bits below
// the segment index, placed in the mantissa of a float in [1, 2), minus 1.
__device__ __forceinline__ float g_lookup(const float4* __restrict__ tab, const TabF32& t, float x) {
  x = fmaxf(x, t.xmin);
  int bits = __float_as_int(x);
  int k = min((bits - t.base) >> t.shift, t.last);
  float v = __int_as_float(((bits << (23 - t.shift)) & 0x007fffff) | 0x3f800000) - 1.0f;
  float4 c = tab[k];
  return fmaf(v, fmaf(v, fmaf(v, c.w, c.z), c.y), c.x);
}

// The FP32 pair kernel keeps a window of the table, from the segment of
// 2^kWinEmin up, in shared memory with every segment stored kRep = 8 times in
// a row (one 128-byte bank row per segment); lane l reads copy l % 8.  The 8
// lanes of a quarter-warp, which share one pass of a 16-byte shared load,
// then always fall in 8 distinct bank groups: the lookups of a warp cost
// four passes whatever segments the lanes hit (a single copy averaged 1.9
// passes per quarter-warp on the 20,000-star field's pairs).  Below 2^kWinEmin
// the argument is clamped: g(x) - g(0) scales as x^(1/3), 2.4e-8 of g(0) there.
constexpr int kWinEmin = -76;
constexpr int kRep = 8;
constexpr int kWinK0 = (kWinEmin - kTabF32.emin) << kTabF32.m;  // first segment kept
constexpr int kWinSegs =  // incl. the zero segment
    ((kTabF32.emax - kTabF32.emin) << kTabF32.m) + 1 - kWinK0;

// tab8 points at copy (lane % 8) of window segment 0.  The window's geometry
// is compile-time, so the segment offset folds into the load's address.
// x must be >= 2^kWinEmin (callers add it to the separation).
constexpr int kWinShift = 23 - kTabF32.m;
constexpr int kWinBaseSeg = (127 + kWinEmin) << kTabF32.m;  // (float bits of 2^kWinEmin) >> shift
constexpr int kWinLast = kWinSegs - 1;
__device__ __forceinline__ float g_lookup_rep(const float4* __restrict__ tab8, float x) {
  const int bits = __float_as_int(x);
  const int k = min((bits >> kWinShift) - kWinBaseSeg, kWinLast);
  const float v = __int_as_float(((bits << (23 - kWinShift)) & 0x007fffff) | 0x3f800000) - 1.0f;
  const float4 c = tab8[k * kRep];
  return fmaf(v, fmaf(v, fmaf(v, c.w, c.z), c.y), c.x);
}

__device__ __forceinline__ double g_lookup(const D4* __restrict__ tab, const TabF64& t,
                                           double x) {
  x = fmax(x, t.xmin);
  int hi = __double2hiint(x);
  int k = min((hi - t.base) >> t.shift, t.last);
  double xlo = __hiloint2double(hi & ~((1 << t.shift) - 1), 0);
  double d = x - xlo;
  const double2* p = reinterpret_cast<const double2*>(tab + k);
  double2 a = __ldg(p), b = __ldg(p + 1);
  return fma(d, fma(d, fma(d, b.y, b.x), a.y), a.x);
}

__device__ __forceinline__ double wendland(double h) {
  if (h >= 1.0) return 0.0;
  double u = 1.0 - h, u2 = u * u;
  return u2 * u2 * (4.0 * h + 1.0);
}
__device__ __forceinline__ float wendland_f(float h) {
  if (h >= 1.0f) return 0.0f;
  const float u = 1.0f - h, u2 = u * u;
  return u2 * u2 * fmaf(4.0f, h, 1.0f);
}

struct QuadParams {
  double inv_L0;
  double inv_cut;
  double log_rho_bar;
  double sigma2;
  int Q;
  int form;
  int taper;
  int symmetric;
};

// One warp per CSR entry (i, j): lanes own the nodes q' of sightline j,
// loop over the nodes q of sightline i, and the warp sums the products.
// In symmetric mode entries with j < i are left for k_mirror.
// Threads per block of the pair kernel: the FP32 form runs one block of 32
// warps per SM around its replicated table (at most 64 registers a thread).
template <typename T, int KPL>
constexpr int pair_threads() { return sizeof(T) == 4 ? (KPL <= 2 ? 1024 : 512) : 256; }

template <typename T, int KPL>
__global__ void __launch_bounds__(pair_threads<T, KPL>()) k_pair_quad(
    QuadParams P, int64_t n_rows, const double* __restrict__ rs, const double* __restrict__ rux,
    const double* __restrict__ ruy, const double* __restrict__ ruz, const double* __restrict__ s,
    const double* __restrict__ ux, const double* __restrict__ uy, const double* __restrict__ uz,
    const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
    T* __restrict__ val, const double* __restrict__ gl_zeta, const double* __restrict__ gl_w,
    const void* __restrict__ gtab, TabF32 tf, TabF64 td, double* __restrict__ kdiag,
    double* __restrict__ prior_m, unsigned* __restrict__ flags, const FieldGrid* __restrict__ fg,
    const int32_t* __restrict__ row_field) {
  extern __shared__ unsigned char smem[];
  typedef typename std::conditional<sizeof(T) == 4, float4, D4>::type T4;
  T* zq = reinterpret_cast<T*>(smem);
  T* wq = zq + kMaxNodes;
  const T4* tab;
  const int lane = threadIdx.x & 31;
  if (sizeof(T) == 4) {
    // the FP32 table window lives in shared memory, kRep copies per segment
    float4* st = reinterpret_cast<float4*>(smem + 2 * kMaxNodes * sizeof(T));
    const float4* gt = reinterpret_cast<const float4*>(gtab) + kWinK0;
    for (int k = threadIdx.x; k < kWinSegs * kRep; k += blockDim.x) st[k] = gt[k / kRep];
    tab = reinterpret_cast<const T4*>(st + (lane & (kRep - 1)));
  } else {
    tab = reinterpret_cast<const T4*>(gtab);
  }
  for (int q = threadIdx.x; q < P.Q; q += blockDim.x) {
    zq[q] = (T)gl_zeta[q];
    wq[q] = (T)gl_w[q];
  }
  __syncthreads();

  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < nnz; e += nwarps) {
    // row of entry e: last r with row_ptr[r] <= e
    int64_t lo = 0, hi = n_rows;
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const int32_t j = col[e];
    if (P.symmetric && j < i) continue;
    const FieldGrid& fgi = fg[row_field ? row_field[i] : 0];
    const double inv_L0 = fgi.inv_L0, inv_cut = fgi.inv_cut;
    const double si = rs[i], sj = s[j];
    const double dx = rux[i] - ux[j], dy = ruy[i] - uy[j], dz = ruz[i] - uz[j];
    const double chord2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const T a = (T)(si * inv_L0), b = (T)(sj * inv_L0), c2 = (T)chord2;
    // this lane's nodes on sightline j
    T tp[KPL], ctp[KPL], wp[KPL];
#pragma unroll
    for (int k = 0; k < KPL; ++k) {
      int q = lane + 32 * k;
      bool ok = q < P.Q;
      tp[k] = ok ? b * zq[q] : (T)0;
      ctp[k] = c2 * tp[k];
      wp[k] = ok ? wq[q] : (T)0;
    }
    T acc = 0;
    for (int q = 0; q < P.Q; ++q) {
      const T t = a * zq[q];
      T inner = 0;
#pragma unroll
      for (int k = 0; k < KPL; ++k) {
        T d = t - tp[k];
        T gv;
        if (sizeof(T) == 4) {
          // x >= 2^kWinEmin by construction: the window's floor is added
          const float x = fmaf((float)d, (float)d,
                               fmaf((float)t, (float)ctp[k], __int_as_float((127 + kWinEmin) << 23)));
          gv = (T)g_lookup_rep(reinterpret_cast<const float4*>(tab), x);
        } else {
          const T x = d * d + t * ctp[k];
          gv = (T)g_lookup(reinterpret_cast<const D4*>(tab), td, (double)x);
        }
        inner += wp[k] * gv;
      }
      acc += wq[q] * inner;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      T K;
      if (sizeof(T) == 4) {
        // FP32 form: the entry's own arithmetic in FP32 too (GB300's FP64
        // pipe is narrow; per-pair FP64 work, not the node sum, bounded this
        // kernel): log1p and the taper to ~1e-7 relative
        const float R = (float)acc;
        float Kf = P.form == GM_FORM_LOGNORMAL ? log1pf(R) : R;
        if (P.taper == GM_TAPER_WENDLAND) {
          // the difference of the distances in FP64: it cancels, and the
          // taper near the cutoff amplifies its error
          const float ds = (float)(si - sj);
          const float d = sqrtf(fmaf(ds, ds, (float)si * (float)sj * (float)c2));
          Kf *= wendland_f(d * (float)inv_cut);
        }
        K = (T)Kf;
      } else {
        const double R = (double)acc;
        double Kd = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
        if (P.taper == GM_TAPER_WENDLAND) {
          const double ds = si - sj;
          const double d = sqrt(fma(ds, ds, si * sj * chord2));
          Kd *= wendland(d * inv_cut);
        }
        K = (T)Kd;
      }
      if (!isfinite((double)K)) atomicOr(flags, kFlagNonFinite);
      val[e] = K;
      if (P.symmetric && j == i) {
        kdiag[i] = (double)K;
        prior_m[i] = P.log_rho_bar + log(si) -
                     (P.form == GM_FORM_LOGNORMAL ? 0.5 * (double)K : 0.5 * P.sigma2);
      }
    }
  }
}

// Lower-triangle entries copy their transpose (rows are sorted).
template <typename T>
__global__ void k_mirror(int64_t n, const int64_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, int64_t nnz, T* __restrict__ val) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int32_t i = (int32_t)lo, j = col[e];
    if (j >= i) continue;
    int64_t a = row_ptr[j], b = row_ptr[j + 1];  // search i in row j
    while (b - a > 1) {
      int64_t mid = (a + b) >> 1;
      if (col[mid] <= i) a = mid; else b = mid;
    }
    val[e] = val[a];
  }
}

// Self-covariance k_qq of query points (FP64, same rule as the diagonal).
template <typename T, int KPL>
__global__ void k_self_quad(QuadParams P, int64_t n_rows, const double* __restrict__ rs,
                            const double* __restrict__ gl_zeta, const double* __restrict__ gl_w,
                            const void* __restrict__ gtab, TabF32 tf, TabF64 td,
                            double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n_rows; r += nwarps) {
    const T a = (T)(rs[r] * P.inv_L0);
    T tp[KPL], wp[KPL];
#pragma unroll
    for (int k = 0; k < KPL; ++k) {
      int q = lane + 32 * k;
      bool ok = q < P.Q;
      tp[k] = ok ? a * (T)gl_zeta[q] : (T)0;
      wp[k] = ok ? (T)gl_w[q] : (T)0;
    }
    T acc = 0;
    for (int q = 0; q < P.Q; ++q) {
      const T t = a * (T)gl_zeta[q];
      T inner = 0;
#pragma unroll
      for (int k = 0; k < KPL; ++k) {
        T d = t - tp[k];
        T x = d * d;
        T gv;
        if (sizeof(T) == 4)
          gv = (T)g_lookup(reinterpret_cast<const float4*>(gtab), tf, (float)x);
        else
          gv = (T)g_lookup(reinterpret_cast<const D4*>(gtab), td, (double)x);
        inner += wp[k] * gv;
      }
      acc += (T)gl_w[q] * inner;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      double R = (double)acc;
      double K = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
      out[r] = (double)(T)K;
    }
  }
}

// ------------------------------------------------------------ band rule
// g by table lookup in the arithmetic type of the inner sums.
template <typename T>
struct GLook;
template <>
struct GLook<float> {
  const float4* tab;
  TabF32 t;
  __device__ float operator()(float x) const { return g_lookup(tab, t, x); }
};
template <>
struct GLook<double> {
  const D4* tab;
  TabF64 t;
  __device__ double operator()(double x) const { return g_lookup(tab, t, x); }
};

// R = I / (s_i s_j) of one pair by the band rule (A = s_i / L0, B = s_j / L0,
// c2 = |u_i - u_j|^2); the warp's lanes share the d-nodes.  Every lane
// returns the sum.
template <typename T>
__device__ __forceinline__ double band_R_warp(double A, double B, double c2, const GLook<T>& g,
                                              int lane) {
  const gmband::Geometry geo = gmband::geometry(A, B, c2);
  T acc = 0;
  const int nk = gmband::d_nodes(geo);
  for (int k = lane; k < nk; k += 32) acc += gmband::d_node<T>(geo, k, g);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return (double)acc / (A * B);
}

template <typename T>
__device__ __forceinline__ GLook<T> band_lookup(const void* gtab, TabF32 tf, TabF64 td,
                                                unsigned char* smem) {
  GLook<T> g;
  if constexpr (sizeof(T) == 4) {
    // the FP32 table lives in shared memory
    float4* st = reinterpret_cast<float4*>(smem);
    const float4* gt = reinterpret_cast<const float4*>(gtab);
    for (int k = threadIdx.x; k <= tf.last; k += blockDim.x) st[k] = gt[k];
    g.tab = st;
    g.t = tf;
  } else {
    g.tab = reinterpret_cast<const D4*>(gtab);
    g.t = td;
  }
  return g;
}

// The band-rule counterpart of k_pair_quad (same entries, taper, mirror
// convention, diagonal and prior mean).
template <typename T>
__global__ void __launch_bounds__(256) k_pair_quad_band(
    QuadParams P, int64_t n_rows, const double* __restrict__ rs, const double* __restrict__ rux,
    const double* __restrict__ ruy, const double* __restrict__ ruz, const double* __restrict__ s,
    const double* __restrict__ ux, const double* __restrict__ uy, const double* __restrict__ uz,
    const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t nnz,
    T* __restrict__ val, const void* __restrict__ gtab, TabF32 tf, TabF64 td,
    double* __restrict__ kdiag, double* __restrict__ prior_m, unsigned* __restrict__ flags,
    const FieldGrid* __restrict__ fg, const int32_t* __restrict__ row_field) {
  extern __shared__ unsigned char smem[];
  const GLook<T> g = band_lookup<T>(gtab, tf, td, smem);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < nnz; e += nwarps) {
    int64_t lo = 0, hi = n_rows;
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const int32_t j = col[e];
    if (P.symmetric && j < i) continue;
    const FieldGrid& fgi = fg[row_field ? row_field[i] : 0];
    const double inv_L0 = fgi.inv_L0, inv_cut = fgi.inv_cut;
    const double si = rs[i], sj = s[j];
    const double dx = rux[i] - ux[j], dy = ruy[i] - uy[j], dz = ruz[i] - uz[j];
    const double chord2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double R = band_R_warp<T>(si * inv_L0, sj * inv_L0, chord2, g, lane);
    if (lane == 0) {
      double K = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
      if (P.taper == GM_TAPER_WENDLAND) {
        double ds = si - sj;
        double d = sqrt(fma(ds, ds, si * sj * chord2));
        K *= wendland(d * inv_cut);
      }
      if (!isfinite(K)) atomicOr(flags, kFlagNonFinite);
      val[e] = (T)K;
      if (P.symmetric && j == i) {
        kdiag[i] = (double)(T)K;
        prior_m[i] = P.log_rho_bar + log(si) -
                     (P.form == GM_FORM_LOGNORMAL ? 0.5 * (double)(T)K : 0.5 * P.sigma2);
      }
    }
  }
}

// Band-rule self-covariance of query points (k_self_quad's counterpart).
template <typename T>
__global__ void __launch_bounds__(256) k_self_quad_band(QuadParams P, int64_t n_rows,
                                                        const double* __restrict__ rs,
                                                        const void* __restrict__ gtab, TabF32 tf,
                                                        TabF64 td, double* __restrict__ out) {
  extern __shared__ unsigned char smem[];
  const GLook<T> g = band_lookup<T>(gtab, tf, td, smem);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n_rows; r += nwarps) {
    const double a = rs[r] * P.inv_L0;
    const double R = band_R_warp<T>(a, a, 0.0, g, lane);
    if (lane == 0) {
      const double K = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
      out[r] = (double)(T)K;
    }
  }
}

// ------------------------------------------------------------ host side
static TabF32 tab_f32() {
  TabF32 t;
  float xmin = ldexpf(1.0f, kTabF32.emin);
  std::memcpy(&t.base, &xmin, sizeof(int));  // bit pattern of 2^emin
  t.shift = 23 - kTabF32.m;
  t.last = kTabF32.n_real();
  t.xmin = xmin;
  return t;
}

static TabF64 tab_f64() {
  TabF64 t;
  double xmin = std::ldexp(1.0, kTabF64.emin);
  long long bits;
  std::memcpy(&bits, &xmin, sizeof(bits));  // bit pattern of 2^emin
  t.base = (int)(bits >> 32);
  t.shift = 20 - kTabF64.m;
  t.last = kTabF64.n_real();
  t.xmin = xmin;
  return t;
}

static const TableGeom& tab_geom(const gm_ctx* c) {
  return c->cfg.precision == GM_PREC_FP32 ? kTabF32 : kTabF64;
}

gm_status phi_points_init(gm_ctx* c) {
  const TableGeom& g = tab_geom(c);
  c->phi_pts = (double*)dev_alloc(c, g.n_pts() * sizeof(double));
  size_t tb = (size_t)(g.n_real() + 1) * (c->cfg.precision == GM_PREC_FP32 ? 16 : 32);
  c->gtab = dev_alloc(c, tb);
  if (!c->phi_pts || !c->gtab) return set_error(c, GM_E_NOMEM, "phi table");
  const double cnorm = std::pow(2.0, 2.0 / 3.0) / std::tgamma(1.0 / 3.0);
  int blocks = (int)std::min<int64_t>(ceil_div(g.n_pts(), 128), 4 * sm_count(c));
  GM_PROF(c, "k_phi_points");
  k_phi_points<<<blocks, 128, 0, c->stream>>>(g, cnorm, c->phi_pts);
  GM_LAUNCH_CHECK(c);
  c->gtab_sigma2 = -1;
  return GM_OK;
}

gm_status gtab_update(gm_ctx* c) {
  if (c->gtab_sigma2 == c->cfg.sigma2 && c->gtab_form == c->cfg.form) return GM_OK;
  const TableGeom& g = tab_geom(c);
  int blocks = (int)std::min<int64_t>(ceil_div(g.n_real() + 1, 256), 4 * sm_count(c));
  GM_PROF(c, "k_gtab");
  if (c->cfg.precision == GM_PREC_FP32)
    k_gtab<float4><<<blocks, 256, 0, c->stream>>>(g, c->phi_pts, c->cfg.sigma2, c->cfg.form, 1,
                                                  (float4*)c->gtab);
  else
    k_gtab<D4><<<blocks, 256, 0, c->stream>>>(g, c->phi_pts, c->cfg.sigma2, c->cfg.form, 0,
                                                   (D4*)c->gtab);
  GM_LAUNCH_CHECK(c);
  c->gtab_sigma2 = c->cfg.sigma2;
  c->gtab_form = c->cfg.form;
  return GM_OK;
}

static QuadParams quad_params(const gm_ctx* c, bool symmetric) {
  QuadParams P;
  P.inv_L0 = 1.0 / c->cfg.outer_scale_pc;
  P.inv_cut = 1.0 / c->cfg.cutoff_pc;
  P.log_rho_bar = std::log(c->cfg.rho_bar);
  P.sigma2 = c->cfg.sigma2;
  P.Q = c->cfg.n_nodes;
  P.form = c->cfg.form;
  P.taper = c->cfg.taper;
  P.symmetric = symmetric ? 1 : 0;
  return P;
}

template <typename T, int KPL>
static void launch_pair(gm_ctx* c, const QuadParams& P, int64_t n_rows, const double* rs,
                        const double* rux, const double* ruy, const double* ruz,
                        const int32_t* row_field, const int64_t* row_ptr, const int32_t* col,
                        int64_t nnz, void* val) {
  size_t smem = 2 * kMaxNodes * sizeof(T);
  if (sizeof(T) == 4) smem += (size_t)kWinSegs * kRep * sizeof(float4);
  constexpr int nt = pair_threads<T, KPL>();
  auto kern = k_pair_quad<T, KPL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  int blocks = std::max(1, per_sm) * sm_count(c);
  blocks = (int)std::min<int64_t>(blocks, std::max<int64_t>(1, ceil_div(nnz * 32, nt)));
  GM_PROF(c, "k_pair_quad");
  kern<<<blocks, nt, smem, c->stream>>>(P, n_rows, rs, rux, ruy, ruz, c->s, c->ux, c->uy, c->uz,
                                         row_ptr, col, nnz, (T*)val, c->gl_zeta, c->gl_w, c->gtab,
                                         tab_f32(), tab_f64(), c->kdiag, c->prior_m, c->d_flags,
                                         c->fgrid, row_field);
}

// Shared memory of the band kernels: the FP32 table (none for FP64).
static size_t band_smem(bool f32) {
  return f32 ? (size_t)(kTabF32.n_real() + 1) * sizeof(float4) : 0;
}

template <typename T>
static void launch_pair_band(gm_ctx* c, const QuadParams& P, int64_t n_rows, const double* rs,
                             const double* rux, const double* ruy, const double* ruz,
                             const int32_t* row_field, const int64_t* row_ptr,
                             const int32_t* col, int64_t nnz, void* val) {
  const size_t smem = band_smem(sizeof(T) == 4);
  auto kern = k_pair_quad_band<T>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  int blocks = std::max(1, per_sm) * sm_count(c);
  blocks = (int)std::min<int64_t>(blocks, std::max<int64_t>(1, ceil_div(nnz * 32, 256)));
  GM_PROF(c, "k_pair_quad_band");
  kern<<<blocks, 256, smem, c->stream>>>(P, n_rows, rs, rux, ruy, ruz, c->s, c->ux, c->uy, c->uz,
                                         row_ptr, col, nnz, (T*)val, c->gtab, tab_f32(),
                                         tab_f64(), c->kdiag, c->prior_m, c->d_flags, c->fgrid,
                                         row_field);
}

gm_status pair_quadrature(gm_ctx* c, int64_t n_rows, const double* rs, const double* rux,
                          const double* ruy, const double* ruz, const int32_t* row_field,
                          const int64_t* row_ptr, const int32_t* col, int64_t nnz, void* val,
                          bool symmetric) {
  if (nnz == 0) return GM_OK;
  gm_status st = gtab_update(c);
  if (st != GM_OK) return st;
  QuadParams P = quad_params(c, symmetric);
  const int Q = c->cfg.n_nodes;
  const bool f32 = c->cfg.precision == GM_PREC_FP32;
  if (c->cfg.quad_rule == GM_QUAD_BAND) {
    if (f32) launch_pair_band<float>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
    else launch_pair_band<double>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
  } else if (Q <= 32) {
    if (f32) launch_pair<float, 1>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
    else launch_pair<double, 1>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
  } else if (Q <= 64) {
    if (f32) launch_pair<float, 2>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
    else launch_pair<double, 2>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
  } else {
    if (f32) launch_pair<float, 4>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
    else launch_pair<double, 4>(c, P, n_rows, rs, rux, ruy, ruz, row_field, row_ptr, col, nnz, val);
  }
  GM_LAUNCH_CHECK(c);
  if (symmetric) {
    int blocks = (int)std::min<int64_t>(ceil_div(nnz, 256), 16 * sm_count(c));
    GM_PROF(c, "k_mirror");
    if (f32) k_mirror<float><<<blocks, 256, 0, c->stream>>>(n_rows, row_ptr, col, nnz, (float*)val);
    else k_mirror<double><<<blocks, 256, 0, c->stream>>>(n_rows, row_ptr, col, nnz, (double*)val);
    GM_LAUNCH_CHECK(c);
  }
  return GM_OK;
}

gm_status mirror_csr(gm_ctx* c, int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t nnz,
                     void* val) {
  if (nnz == 0) return GM_OK;
  int blocks = (int)std::min<int64_t>(ceil_div(nnz, 256), 16 * sm_count(c));
  GM_PROF(c, "k_mirror");
  if (c->cfg.precision == GM_PREC_FP32)
    k_mirror<float><<<blocks, 256, 0, c->stream>>>(n, row_ptr, col, nnz, (float*)val);
  else
    k_mirror<double><<<blocks, 256, 0, c->stream>>>(n, row_ptr, col, nnz, (double*)val);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status self_quadrature(gm_ctx* c, int64_t n_rows, const double* rs, double* kss) {
  if (n_rows == 0) return GM_OK;
  gm_status st = gtab_update(c);
  if (st != GM_OK) return st;
  QuadParams P = quad_params(c, false);
  const int Q = c->cfg.n_nodes;
  const bool f32 = c->cfg.precision == GM_PREC_FP32;
  int blocks = (int)std::min<int64_t>(ceil_div(n_rows * 32, 256), 8 * sm_count(c));
  if (c->cfg.quad_rule == GM_QUAD_BAND) {
    const size_t smem = band_smem(f32);
    GM_PROF(c, "k_self_quad_band");
    if (f32) {
      cudaFuncSetAttribute(k_self_quad_band<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      k_self_quad_band<float><<<blocks, 256, smem, c->stream>>>(P, n_rows, rs, c->gtab,
                                                                tab_f32(), tab_f64(), kss);
    } else {
      k_self_quad_band<double><<<blocks, 256, 0, c->stream>>>(P, n_rows, rs, c->gtab, tab_f32(),
                                                              tab_f64(), kss);
    }
    GM_LAUNCH_CHECK(c);
    return GM_OK;
  }
#define GM_SELF(T, K)                                                                     \
  k_self_quad<T, K><<<blocks, 256, 0, c->stream>>>(P, n_rows, rs, c->gl_zeta, c->gl_w, \
                                                    c->gtab, tab_f32(), tab_f64(), kss)
  GM_PROF(c, "k_self_quad");
  if (Q <= 32) {
    if (f32) GM_SELF(float, 1); else GM_SELF(double, 1);
  } else if (Q <= 64) {
    if (f32) GM_SELF(float, 2); else GM_SELF(double, 2);
  } else {
    if (f32) GM_SELF(float, 4); else GM_SELF(double, 4);
  }
#undef GM_SELF
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm

namespace gm {

// Sightline quadrature for an explicit list of pair geometries (distances
// si, sj in pc, chord |u_i - u_j|): K = log1p(R) (or R) without the taper.
// Same rule and kernel table as the covariance assembly; one warp per pair.
template <typename T, int KPL>
__global__ void __launch_bounds__(256) k_pairlist_quad(
    QuadParams P, int64_t n, const double* __restrict__ si, const double* __restrict__ sj,
    const double* __restrict__ chord, double* __restrict__ out,
    const double* __restrict__ gl_zeta, const double* __restrict__ gl_w,
    const void* __restrict__ gtab, TabF32 tf, TabF64 td) {
  extern __shared__ unsigned char smem[];
  typedef typename std::conditional<sizeof(T) == 4, float4, D4>::type T4;
  T* zq = reinterpret_cast<T*>(smem);
  T* wq = zq + kMaxNodes;
  const T4* tab;
  if (sizeof(T) == 4) {
    float4* st = reinterpret_cast<float4*>(smem + 2 * kMaxNodes * sizeof(T));
    const float4* gt = reinterpret_cast<const float4*>(gtab);
    for (int k = threadIdx.x; k <= tf.last; k += blockDim.x) st[k] = gt[k];
    tab = reinterpret_cast<const T4*>(st);
  } else {
    tab = reinterpret_cast<const T4*>(gtab);
  }
  for (int q = threadIdx.x; q < P.Q; q += blockDim.x) {
    zq[q] = (T)gl_zeta[q];
    wq[q] = (T)gl_w[q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < n; p += nwarps) {
    const T a = (T)(si[p] * P.inv_L0), b = (T)(sj[p] * P.inv_L0);
    const T c2 = (T)(chord[p] * chord[p]);
    T tp[KPL], ctp[KPL], wp[KPL];
#pragma unroll
    for (int k = 0; k < KPL; ++k) {
      int q = lane + 32 * k;
      bool ok = q < P.Q;
      tp[k] = ok ? b * zq[q] : (T)0;
      ctp[k] = c2 * tp[k];
      wp[k] = ok ? wq[q] : (T)0;
    }
    T acc = 0;
    for (int q = 0; q < P.Q; ++q) {
      const T t = a * zq[q];
      T inner = 0;
#pragma unroll
      for (int k = 0; k < KPL; ++k) {
        T d = t - tp[k];
        T x = d * d + t * ctp[k];
        T gv;
        if (sizeof(T) == 4)
          gv = (T)g_lookup(reinterpret_cast<const float4*>(tab), tf, (float)x);
        else
          gv = (T)g_lookup(reinterpret_cast<const D4*>(tab), td, (double)x);
        inner += wp[k] * gv;
      }
      acc += wq[q] * inner;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      const double R = (double)acc;
      out[p] = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
    }
  }
}

// Band-rule counterpart of k_pairlist_quad.
template <typename T>
__global__ void __launch_bounds__(256) k_pairlist_quad_band(
    QuadParams P, int64_t n, const double* __restrict__ si, const double* __restrict__ sj,
    const double* __restrict__ chord, double* __restrict__ out, const void* __restrict__ gtab,
    TabF32 tf, TabF64 td) {
  extern __shared__ unsigned char smem[];
  const GLook<T> g = band_lookup<T>(gtab, tf, td, smem);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < n; p += nwarps) {
    const double R = band_R_warp<T>(si[p] * P.inv_L0, sj[p] * P.inv_L0, chord[p] * chord[p], g,
                                    lane);
    if (lane == 0) out[p] = P.form == GM_FORM_LOGNORMAL ? log1p(R) : R;
  }
}

template <typename T>
static void launch_pairlist_band(gm_ctx* c, const QuadParams& P, int64_t n, const double* si,
                                 const double* sj, const double* chord, double* out) {
  const size_t smem = band_smem(sizeof(T) == 4);
  auto kern = k_pairlist_quad_band<T>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  int blocks = std::max(1, per_sm) * sm_count(c);
  blocks = (int)std::min<int64_t>(blocks, std::max<int64_t>(1, ceil_div(n * 32, 256)));
  kern<<<blocks, 256, smem, c->stream>>>(P, n, si, sj, chord, out, c->gtab, tab_f32(),
                                         tab_f64());
}

template <typename T, int KPL>
static void launch_pairlist(gm_ctx* c, const QuadParams& P, int64_t n, const double* si,
                            const double* sj, const double* chord, double* out) {
  size_t smem = 2 * kMaxNodes * sizeof(T);
  if (sizeof(T) == 4) smem += (size_t)(kTabF32.n_real() + 1) * sizeof(float4);
  auto kern = k_pairlist_quad<T, KPL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  int blocks = std::max(1, per_sm) * sm_count(c);
  blocks = (int)std::min<int64_t>(blocks, std::max<int64_t>(1, ceil_div(n * 32, 256)));
  kern<<<blocks, 256, smem, c->stream>>>(P, n, si, sj, chord, out, c->gl_zeta, c->gl_w, c->gtab,
                                         tab_f32(), tab_f64());
}

gm_status pairlist_quadrature(gm_ctx* c, int64_t n, const double* si, const double* sj,
                              const double* chord, double* out) {
  if (n == 0) return GM_OK;
  gm_status st = gtab_update(c);
  if (st != GM_OK) return st;
  QuadParams P = quad_params(c, false);
  const int Q = c->cfg.n_nodes;
  const bool f32 = c->cfg.precision == GM_PREC_FP32;
  if (c->cfg.quad_rule == GM_QUAD_BAND) {
    GM_PROF(c, "k_pairlist_quad_band");
    if (f32) launch_pairlist_band<float>(c, P, n, si, sj, chord, out);
    else launch_pairlist_band<double>(c, P, n, si, sj, chord, out);
    GM_LAUNCH_CHECK(c);
    return GM_OK;
  }
  GM_PROF(c, "k_pairlist_quad");
  if (Q <= 32) {
    if (f32) launch_pairlist<float, 1>(c, P, n, si, sj, chord, out);
    else launch_pairlist<double, 1>(c, P, n, si, sj, chord, out);
  } else if (Q <= 64) {
    if (f32) launch_pairlist<float, 2>(c, P, n, si, sj, chord, out);
    else launch_pairlist<double, 2>(c, P, n, si, sj, chord, out);
  } else {
    if (f32) launch_pairlist<float, 4>(c, P, n, si, sj, chord, out);
    else launch_pairlist<double, 4>(c, P, n, si, sj, chord, out);
  }
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm
