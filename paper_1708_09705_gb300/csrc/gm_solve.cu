// Posterior marginals of the EP approximation by sparse solves.
//
// With site precisions tau (S = diag tau, D = S^1/2) and natural means nu, the
// posterior is N(mu, Sigma) with Sigma = (K^-1 + S)^-1.  Written as the noisy-GP
// conditional of Sect. 2 (eq. cond_GP0) with noise 1/tau, and through the
// well-conditioned B = I + D K D (eigenvalues >= 1, valid for tau_i = 0):
//   b = nu - tau o m,  B y = D K b,  alpha = b - D y,  mu = m + K alpha,
//   Sigma_ii = K_ii - v_i^T B^-1 v_i,  v_i = D K e_i  (column i of K, scaled).
// B is applied matrix-free from the CSR of K.  The mean needs one solve; the
// variances need one per star and run as panels of many right-hand sides that
// share every matrix read.  All solves are Jacobi-preconditioned CG
// (M = diag B = 1 + tau_i K_ii).  In FP32 mode the mean solve is refined in
// FP64: residuals b - B x are recomputed in FP64 and FP32 CG solves for the
// correction.  Reductions use per-block partials summed in a fixed order, so
// reruns are bit-identical.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

struct Workspace {
  Buffer b64, w64, x64, r64, d64, minv64, dx64, kdx64;  // FP64 vectors
  Buffer r32;                                          // FP32 refinement residual
  Buffer x, r, p, pd, q, dv, minv;                    // solver-precision vectors
  Buffer part;                                        // block partials (single RHS)
  Buffer P_X, P_R, P_P, P_PD, P_Q;                    // panels n x R
  Buffer P_part, P_scal, P_active;                    // panel partials / scalars
};

void workspace_free(gm_ctx* c) {
  delete c->ws;
  c->ws = nullptr;
}

static Workspace& W(gm_ctx* c) {
  if (!c->ws) c->ws = new Workspace();
  return *c->ws;
}

constexpr int kBT = 256;  // threads per block of the vector kernels

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block sum of one double per thread (fixed order), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// Sum of a partials array, same fixed order in every block.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int n, double* sh) {
  double v = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  double t = block_sum(v, sh);
  if (threadIdx.x == 0) sh[32] = t;
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- SpMV
// Row dot products of the CSR of K are HBM-bound: per stored entry a 4-byte
// column index and a 4- or 8-byte value are streamed once, and the gathered
// x[col] hits L1/L2.  A warp owns a row; each lane loads 16-byte vectors of
// values and column indices (float4 + int4, or double2 + int2) over the
// 16-byte-aligned body of the row, two vectors in flight per iteration, with
// the ragged head and tail of the row loaded as scalars.  The value and index
// streams are read with the evict-first hint so that x stays in L1.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; using C = int4; };
template <> struct Vec16<double> { using V = double2; using C = int2; };

template <typename TAcc, typename TX>
__device__ __forceinline__ TAcc vdot(const float4 v, const int4 c, const TX* __restrict__ x) {
  return (TAcc)v.x * (TAcc)x[c.x] + (TAcc)v.y * (TAcc)x[c.y] + (TAcc)v.z * (TAcc)x[c.z] +
         (TAcc)v.w * (TAcc)x[c.w];
}
template <typename TAcc, typename TX>
__device__ __forceinline__ TAcc vdot(const double2 v, const int2 c, const TX* __restrict__ x) {
  return (TAcc)v.x * (TAcc)x[c.x] + (TAcc)v.y * (TAcc)x[c.y];
}

// This lane's share of sum_{e in [b, e1)} val[e] x[col[e]].
template <typename TAcc, typename TA, typename TX>
__device__ __forceinline__ TAcc row_dot_lane(int64_t b, int64_t e1, const int32_t* __restrict__ col,
                                             const TA* __restrict__ val,
                                             const TX* __restrict__ x, int lane) {
  constexpr int V = 16 / sizeof(TA);
  using VA = typename Vec16<TA>::V;
  using VC = typename Vec16<TA>::C;
  TAcc acc = 0;
  int64_t a = (b + V - 1) / V * V;  // first vector-aligned entry of the row
  if (a > e1) a = e1;
  if (b + lane < a) acc += (TAcc)__ldcs(val + b + lane) * (TAcc)x[__ldcs(col + b + lane)];
  const int64_t ng = (e1 - a) / V;
  const VA* va = reinterpret_cast<const VA*>(val + a);
  const VC* vc = reinterpret_cast<const VC*>(col + a);
  int64_t k = lane;
  for (; k + 32 < ng; k += 64) {
    const VA v0 = __ldcs(va + k), v1 = __ldcs(va + k + 32);
    const VC c0 = __ldcs(vc + k), c1 = __ldcs(vc + k + 32);
    acc += vdot<TAcc>(v0, c0, x);
    acc += vdot<TAcc>(v1, c1, x);
  }
  if (k < ng) acc += vdot<TAcc>(__ldcs(va + k), __ldcs(vc + k), x);
  const int64_t t = a + ng * V;
  if (t + lane < e1) acc += (TAcc)__ldcs(val + t + lane) * (TAcc)x[__ldcs(col + t + lane)];
  return acc;
}

// y = K x (FP64 accumulate), optionally y = base + K x.  Warp per row.
// val and col must be 16-byte aligned (every device buffer of the library is).
template <typename TA, typename TX>
__global__ void k_spmv(int64_t n_rows, const int64_t* __restrict__ row_ptr,
                       const int32_t* __restrict__ col, const TA* __restrict__ val,
                       const TX* __restrict__ x, const double* __restrict__ base,
                       double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n_rows; i += nw) {
    double acc = row_dot_lane<double>(row_ptr[i], row_ptr[i + 1], col, val, x, lane);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = (base ? base[i] : 0.0) + acc;
  }
}

// q = p + d o (K pd), pq partial.  Warp per row; kBTB threads per block so
// that the grid of the CG vector kernels (2 blocks per SM) keeps 32 warps of
// loads in flight on every SM.
constexpr int kBTB = 512;
template <typename TA, typename TV>
__global__ void __launch_bounds__(kBTB) k_apply_B(int64_t n, const int64_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col,
                                                  const TA* __restrict__ val,
                                                  const TV* __restrict__ dv,
                                                  const TV* __restrict__ p,
                                                  const TV* __restrict__ pd, TV* __restrict__ q,
                                                  double* __restrict__ pq_part) {
  __shared__ double sh[40];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double pq = 0;
  for (int64_t i = warp; i < n; i += nw) {
    TV acc = row_dot_lane<TV>(row_ptr[i], row_ptr[i + 1], col, val, pd, lane);
    acc = warp_sum(acc);
    if (lane == 0) {
      TV qi = p[i] + dv[i] * acc;
      q[i] = qi;
      pq += (double)p[i] * (double)qi;
    }
  }
  double t = block_sum(pq, sh);
  if (threadIdx.x == 0) pq_part[blockIdx.x] = t;
}

// Partials layout for single-RHS CG (G = gridDim of the vector kernels):
// [0,G) pq, [G,2G) rz even, [2G,3G) rz odd, [3G,4G) rr, [4G,5G) bb.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_cg_init(int64_t n, const TV* __restrict__ rhs,
                                                 const TV* __restrict__ minv,
                                                 const TV* __restrict__ dv, TV* __restrict__ x,
                                                 TV* __restrict__ r, TV* __restrict__ p,
                                                 TV* __restrict__ pd, double* __restrict__ part) {
  __shared__ double sh[40];
  const int G = gridDim.x;
  double rz = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)G * blockDim.x) {
    TV ri = rhs[i];
    TV zi = minv[i] * ri;
    x[i] = 0;
    r[i] = ri;
    p[i] = zi;
    pd[i] = dv[i] * zi;
    rz += (double)ri * (double)zi;
    bb += (double)ri * (double)ri;
  }
  double a = block_sum(rz, sh);
  double b2 = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    part[G + blockIdx.x] = a;       // rz "previous" slot of iteration 1 (even)
    part[3 * G + blockIdx.x] = b2;  // rr = bb at start
    part[4 * G + blockIdx.x] = b2;
  }
}

// Iteration it (1-based): alpha = rz_prev / pq; x += alpha p; r -= alpha q;
// rz_new = r . M^-1 r into the other parity slot, rr = r . r.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_cg_update1(int64_t n, int it, const TV* __restrict__ minv,
                                                    TV* __restrict__ x, TV* __restrict__ r,
                                                    const TV* __restrict__ p,
                                                    const TV* __restrict__ q,
                                                    double* __restrict__ part,
                                                    unsigned* __restrict__ flags) {
  __shared__ double sh[40];
  const int G = gridDim.x;
  const int prev = (it & 1) ? 1 : 2, next = (it & 1) ? 2 : 1;
  double pq = sum_partials(part, G, sh);
  double rzp = sum_partials(part + prev * G, G, sh);
  double alpha = 0;
  if (rzp > 0) {
    if (pq > 0) alpha = rzp / pq;
    else if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, kFlagNotSPD);
  }
  const TV a = (TV)alpha;
  double rz = 0, rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)G * blockDim.x) {
    x[i] += a * p[i];
    TV ri = r[i] - a * q[i];
    r[i] = ri;
    rz += (double)ri * (double)(minv[i] * ri);
    rr += (double)ri * (double)ri;
  }
  double t1 = block_sum(rz, sh);
  double t2 = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    part[next * G + blockIdx.x] = t1;
    part[3 * G + blockIdx.x] = t2;
  }
}

// beta = rz_new / rz_prev; p = M^-1 r + beta p; pd = d o p.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_cg_update2(int64_t n, int it, const TV* __restrict__ minv,
                                                    const TV* __restrict__ dv,
                                                    const TV* __restrict__ r, TV* __restrict__ p,
                                                    TV* __restrict__ pd,
                                                    const double* __restrict__ part) {
  __shared__ double sh[40];
  const int G = gridDim.x;
  const int prev = (it & 1) ? 1 : 2, next = (it & 1) ? 2 : 1;
  double rzp = sum_partials(part + prev * G, G, sh);
  double rzn = sum_partials(part + next * G, G, sh);
  const TV beta = (TV)(rzp > 0 ? rzn / rzp : 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)G * blockDim.x) {
    TV pi = minv[i] * r[i] + beta * p[i];
    p[i] = pi;
    pd[i] = dv[i] * pi;
  }
}

// ---------------------------------------------------------------- elementwise
__global__ void k_site_rhs(int64_t n, const double* __restrict__ nu, const double* __restrict__ tau,
                           const double* __restrict__ m, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = nu[i] - tau[i] * m[i];
}

template <typename TV>
__global__ void k_precond(int64_t n, const double* __restrict__ tau,
                          const double* __restrict__ kdiag, TV* __restrict__ dv,
                          TV* __restrict__ minv, double* __restrict__ d64,
                          double* __restrict__ minv64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = sqrt(fmax(tau[i], 0.0));
    double mi = 1.0 / (1.0 + tau[i] * kdiag[i]);
    dv[i] = (TV)d;
    minv[i] = (TV)mi;
    d64[i] = d;
    minv64[i] = mi;
  }
}

// out = scale_a o a (+ add)  helpers
template <typename TO>
__global__ void k_scale(int64_t n, const double* __restrict__ d, const double* __restrict__ a,
                        TO* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)(d[i] * a[i]);
}

// alpha = b - d o y
template <typename TY>
__global__ void k_alpha(int64_t n, const double* __restrict__ b, const double* __restrict__ d,
                        const TY* __restrict__ y, double* __restrict__ alpha) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    alpha[i] = b[i] - d[i] * (double)y[i];
}

// FP64 residual of B x = rhs: r = rhs - x - d o (K (d o x)); also x (FP64) += e.
__global__ void k_refine_add(int64_t n, double* __restrict__ x64, const float* __restrict__ e,
                             const double* __restrict__ d, double* __restrict__ dx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double xi = x64[i] + (double)e[i];
    x64[i] = xi;
    dx[i] = d[i] * xi;
  }
}

__global__ void __launch_bounds__(kBT) k_refine_resid(int64_t n, const double* __restrict__ rhs,
                                                      const double* __restrict__ x64,
                                                      const double* __restrict__ d,
                                                      const double* __restrict__ kdx,
                                                      double* __restrict__ r64,
                                                      float* __restrict__ r32,
                                                      double* __restrict__ part) {
  __shared__ double sh[40];
  double rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ri = rhs[i] - x64[i] - d[i] * kdx[i];
    r64[i] = ri;
    r32[i] = (float)ri;
    rr += ri * ri;
    bb += rhs[i] * rhs[i];
  }
  double a = block_sum(rr, sh);
  double b = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
  }
}

// ---------------------------------------------------------------- panels
// Panel arrays are n x R row-major (R a multiple of 32).  Grid: x over rows
// (warp-strided), y over 32-column chunks; lane = column within the chunk.
// Column partials: part[(bx) * R + c].

// Right-hand sides scattered from CSR rows (rows of K for the stars, query
// rows for prediction).  Column c solves for row r = r0 + c:
//   v_r = d o k_r                  (k_rr - v_r^T B^-1 v_r = Sigma_rr), or, for
//   e_r when `unit` marks r        ((B^-1)_rr = y_r, Sigma_rr = (1 - y_r) / tau_r).
// The unit form is used for stars whose own site dominates (tau_r K_rr >= 1):
// there the cavity precision tau_r y_r / (1 - y_r) keeps the relative accuracy
// of y_r, whereas 1/Sigma_rr - tau_r would cancel.
__device__ __forceinline__ bool unit_rhs(const double* __restrict__ tau,
                                         const double* __restrict__ kd, int64_t r) {
  return tau != nullptr && tau[r] * kd[r] >= 1.0;
}

template <typename TA, typename TV>
__global__ void k_panel_rhs(int64_t r0, int64_t n_cols, int R, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const TA* __restrict__ val,
                            const TV* __restrict__ dv, const double* __restrict__ tau,
                            const double* __restrict__ kd, TV* __restrict__ Rr) {
  // one warp per right-hand side
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < n_cols; c += nw) {
    const int64_t r = r0 + c;
    if (unit_rhs(tau, kd, r)) {
      if (lane == 0) Rr[r * R + c] = (TV)1;
      continue;
    }
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
      int32_t j = col[e];
      Rr[(int64_t)j * R + c] = dv[j] * (TV)val[e];
    }
  }
}

// Probed right-hand sides: column k sums the right-hand sides of the stars of
// colour class c0 + k (v_r or e_r as above).  One thread per row j, so that
// every panel entry is summed in a fixed order: (j, colour(r)) receives
// d_j K_jr for each non-unit neighbour r of j, and (j, colour(j)) receives 1
// when j itself is a unit star.
template <typename TA, typename TV>
__global__ void k_panel_rhs_probe(int64_t n, int64_t c0, int64_t n_cols, int R,
                                  const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col, const TA* __restrict__ val,
                                  const TV* __restrict__ dv, const double* __restrict__ tau,
                                  const double* __restrict__ kd, const int32_t* __restrict__ pcol,
                                  TV* __restrict__ Rr) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    TV* row = Rr + j * R;
    const TV dj = dv[j];
    for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
      const int32_t r = col[e];
      const int64_t k = (int64_t)pcol[r] - c0;
      if (k < 0 || k >= n_cols || unit_rhs(tau, kd, r)) continue;
      row[k] += dj * (TV)val[e];
    }
    const int64_t kj = (int64_t)pcol[j] - c0;
    if (kj >= 0 && kj < n_cols && unit_rhs(tau, kd, j)) row[kj] += (TV)1;
  }
}

// The same with a warp per row j, for colourings at least 2 x cutoff apart:
// two neighbours of j are then within 2 x cutoff of each other, so they have
// distinct colours and every entry of the row is written once (the adds go to
// zeroed entries and give the same bits as the loop above; an add is used
// all the same, so that a collision at the rounding edge of the separation
// test would still sum).  The lanes share the row's neighbour list.
template <typename TA, typename TV>
__global__ void k_panel_rhs_probe_w(int64_t n, int64_t c0, int64_t n_cols, int R,
                                    const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col, const TA* __restrict__ val,
                                    const TV* __restrict__ dv, const double* __restrict__ tau,
                                    const double* __restrict__ kd,
                                    const int32_t* __restrict__ pcol, TV* __restrict__ Rr) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < n; j += nw) {
    TV* row = Rr + j * R;
    const TV dj = dv[j];
    for (int64_t e = row_ptr[j] + lane; e < row_ptr[j + 1]; e += 32) {
      const int32_t r = col[e];
      const int64_t k = (int64_t)pcol[r] - c0;
      if (k < 0 || k >= n_cols || unit_rhs(tau, kd, r)) continue;
      atomicAdd(row + k, dj * (TV)val[e]);
    }
    if (lane == 0) {
      const int64_t kj = (int64_t)pcol[j] - c0;
      if (kj >= 0 && kj < n_cols && unit_rhs(tau, kd, j)) atomicAdd(row + kj, (TV)1);
    }
  }
}

template <typename TV>
__global__ void __launch_bounds__(kBT) k_panel_init(int64_t n, int R, const TV* __restrict__ minv,
                                                    const TV* __restrict__ dv,
                                                    TV* __restrict__ X, const TV* __restrict__ Rr,
                                                    TV* __restrict__ P, TV* __restrict__ PD,
                                                    double* __restrict__ part_rz,
                                                    double* __restrict__ part_bb) {
  __shared__ double sh_rz[8][32], sh_bb[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  PartialSum<TV> rz, bb;
  for (int64_t i = w; i < n; i += nw) {
    int64_t k = i * R + c;
    TV ri = Rr[k];
    TV zi = minv[i] * ri;
    X[k] = 0;
    P[k] = zi;
    PD[k] = dv[i] * zi;
    rz.add(ri * zi);
    bb.add(ri * ri);
  }
  sh_rz[wib][lane] = rz.value();
  sh_bb[wib][lane] = bb.value();
  __syncthreads();
  if (wib == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh_rz[k][lane];
      b += sh_bb[k][lane];
    }
    part_rz[(int64_t)blockIdx.x * R + c] = a;
    part_bb[(int64_t)blockIdx.x * R + c] = b;
  }
}

// Warm start: PD = d o X (so that the panel product gives Q = B X).
template <typename TV>
__global__ void __launch_bounds__(kBT) k_panel_scale(int64_t n, int R, const TV* __restrict__ dv,
                                                     const TV* __restrict__ X, TV* __restrict__ PD) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = w; i < n; i += nw) {
    int64_t k = i * R + c;
    PD[k] = dv[i] * X[k];
  }
}

// Warm start: with Rr = v (the right-hand sides) and Q = B X0, set the
// residual Rr = v - Q, P = M^-1 Rr, PD = d o P; partial rz and ||v||^2.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_panel_init_warm(int64_t n, int R, const TV* __restrict__ minv,
                                                         const TV* __restrict__ dv,
                                                         TV* __restrict__ Rr, const TV* __restrict__ Q,
                                                         TV* __restrict__ P, TV* __restrict__ PD,
                                                         double* __restrict__ part_rz,
                                                         double* __restrict__ part_bb) {
  __shared__ double sh_rz[8][32], sh_bb[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  PartialSum<TV> rz, bb;
  for (int64_t i = w; i < n; i += nw) {
    int64_t k = i * R + c;
    TV v = Rr[k];
    TV ri = v - Q[k];
    TV zi = minv[i] * ri;
    Rr[k] = ri;
    P[k] = zi;
    PD[k] = dv[i] * zi;
    rz.add(ri * zi);
    bb.add(v * v);
  }
  sh_rz[wib][lane] = rz.value();
  sh_bb[wib][lane] = bb.value();
  __syncthreads();
  if (wib == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh_rz[k][lane];
      b += sh_bb[k][lane];
    }
    part_rz[(int64_t)blockIdx.x * R + c] = a;
    part_bb[(int64_t)blockIdx.x * R + c] = b;
  }
}

// Q = P + d o (K PD), partial pq per column.  Warp per (row, chunk); the
// row's (col, val) pairs are loaded 32 at a time and broadcast by shuffle.
template <typename TA, typename TV>
__global__ void __launch_bounds__(kBT) k_panel_spmm(int64_t n, int R,
                                                    const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col,
                                                    const TA* __restrict__ val,
                                                    const TV* __restrict__ dv,
                                                    const TV* __restrict__ P,
                                                    const TV* __restrict__ PD, TV* __restrict__ Q,
                                                    double* __restrict__ part_pq) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  PartialSum<TV> pq;
  for (int64_t i = w; i < n; i += nw) {
    const int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
    TV acc = 0;
    for (int64_t eb = e0; eb < e1; eb += 32) {
      int32_t jl = 0;
      TV vl = 0;
      if (eb + lane < e1) {
        jl = col[eb + lane];
        vl = (TV)val[eb + lane];
      }
      const int cnt = (e1 - eb) < 32 ? (int)(e1 - eb) : 32;
      for (int k = 0; k < cnt; ++k) {
        int32_t j = __shfl_sync(0xffffffffu, jl, k);
        TV v = __shfl_sync(0xffffffffu, vl, k);
        acc += v * PD[(int64_t)j * R + c];
      }
    }
    const int64_t k = i * R + c;
    TV pi = P[k];
    TV qi = pi + dv[i] * acc;
    Q[k] = qi;
    pq.add(pi * qi);
  }
  sh[wib][lane] = pq.value();
  __syncthreads();
  if (wib == 0) {
    double a = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += sh[k][lane];
    part_pq[(int64_t)blockIdx.x * R + c] = a;
  }
}

// Per-column sums of partials.  scal layout (R each): 0 alpha, 1 beta,
// 2 rz_prev, 3 rz_new, 4 bb, 5 rr.  mode 0: after init (rz_prev, bb);
// mode 1: after spmm (alpha); mode 2: after update1 (beta, activity).
// corr: ncorr more rows added to the pa sums (the deflation term of r^T z).
__global__ void k_panel_reduce(int mode, int nbx, int R, int64_t n_cols, double tol2, int it,
                               int max_it, const double* __restrict__ pa,
                               const double* __restrict__ pb, const double* __restrict__ corr,
                               int ncorr, double* __restrict__ scal, int* __restrict__ active,
                               int* __restrict__ n_active, unsigned* __restrict__ flags) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    double a = 0, b = 0;
    for (int k = 0; k < nbx; ++k) {
      a += pa[(int64_t)k * R + c];
      if (pb) b += pb[(int64_t)k * R + c];
    }
    for (int k = 0; k < ncorr; ++k) a += corr[(int64_t)k * R + c];
    double* alpha = scal;
    double* beta = scal + R;
    double* rzp = scal + 2 * R;
    double* rzn = scal + 3 * R;
    double* bb = scal + 4 * R;
    double* rr = scal + 5 * R;
    if (mode == 0) {
      rzp[c] = a;
      bb[c] = b;
      rr[c] = b;
      int act = (c < n_cols) && (b > 0);
      active[c] = act;
      if (act) atomicAdd(n_active, 1);
    } else if (mode == 1) {
      double al = 0;
      if (active[c]) {
        if (a > 0 && rzp[c] > 0) al = rzp[c] / a;
        else if (rzp[c] > 0) {
          atomicOr(flags, kFlagNotSPD);
          active[c] = 0;
        }
      }
      alpha[c] = al;
    } else {
      rzn[c] = a;
      rr[c] = b;
      double be = 0;
      if (active[c]) {
        if (!isfinite(a) || !isfinite(b)) {
          atomicOr(flags, kFlagNonFinite);
          active[c] = 0;
        } else if (b <= tol2 * bb[c] || it >= max_it) {
          active[c] = 0;
        } else {
          be = rzp[c] > 0 ? a / rzp[c] : 0.0;
          atomicAdd(n_active, 1);
        }
      }
      beta[c] = be;
      rzp[c] = a;
    }
  }
}

// X += alpha P, Rr -= alpha Q, partial rz (with M^-1) and rr.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_panel_update1(int64_t n, int R, const TV* __restrict__ minv,
                                                       const double* __restrict__ scal,
                                                       TV* __restrict__ X, TV* __restrict__ Rr,
                                                       const TV* __restrict__ P,
                                                       const TV* __restrict__ Q,
                                                       double* __restrict__ part_rz,
                                                       double* __restrict__ part_rr) {
  __shared__ double sh_a[8][32], sh_b[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const TV a = (TV)scal[c];
  PartialSum<TV> rz, rr;
  // four rows per pass with all loads issued first (memory-level parallelism)
  int64_t i = w;
  for (; i + 3 * nw < n; i += 4 * nw) {
    TV x[4], p[4], r[4], q[4], m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = (i + u * nw) * R + c;
      x[u] = X[k];
      p[u] = P[k];
      r[u] = Rr[k];
      q[u] = Q[k];
      m[u] = minv[i + u * nw];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = (i + u * nw) * R + c;
      X[k] = x[u] + a * p[u];
      const TV ri = r[u] - a * q[u];
      Rr[k] = ri;
      rz.add(ri * (m[u] * ri));
      rr.add(ri * ri);
    }
  }
  for (; i < n; i += nw) {
    int64_t k = i * R + c;
    X[k] += a * P[k];
    TV ri = Rr[k] - a * Q[k];
    Rr[k] = ri;
    rz.add(ri * (minv[i] * ri));
    rr.add(ri * ri);
  }
  sh_a[wib][lane] = rz.value();
  sh_b[wib][lane] = rr.value();
  __syncthreads();
  if (wib == 0) {
    double s1 = 0, s2 = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s1 += sh_a[k][lane];
      s2 += sh_b[k][lane];
    }
    part_rz[(int64_t)blockIdx.x * R + c] = s1;
    part_rr[(int64_t)blockIdx.x * R + c] = s2;
  }
}

// P = M^-1 Rr + beta P (active columns), PD = d o P.
template <typename TV>
__global__ void __launch_bounds__(kBT) k_panel_update2(int64_t n, int R, const TV* __restrict__ minv,
                                                       const TV* __restrict__ dv,
                                                       const double* __restrict__ scal,
                                                       const int* __restrict__ active,
                                                       const TV* __restrict__ Rr,
                                                       TV* __restrict__ P, TV* __restrict__ PD) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  if (!active[c]) return;  // frozen column: P is never read with alpha != 0
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const TV be = (TV)scal[R + c];
  int64_t i = w;
  for (; i + 3 * nw < n; i += 4 * nw) {
    TV r[4], p[4], m[4], d[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = (i + u * nw) * R + c;
      r[u] = Rr[k];
      p[u] = P[k];
      m[u] = minv[i + u * nw];
      d[u] = dv[i + u * nw];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = (i + u * nw) * R + c;
      const TV pi = m[u] * r[u] + be * p[u];
      P[k] = pi;
      PD[k] = d[u] * pi;
    }
  }
  for (; i < n; i += nw) {
    int64_t k = i * R + c;
    TV pi = minv[i] * Rr[k] + be * P[k];
    P[k] = pi;
    PD[k] = dv[i] * pi;
  }
}

// Sigma_rr from the solution column: k_rr - v_r^T y (v_r = d o k_r) or
// (1 - y_r) / tau_r for unit right-hand sides.
template <typename TA, typename TV>
__global__ void k_panel_final(int64_t r0, int64_t n_cols, int R, const int64_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, const TA* __restrict__ val,
                              const double* __restrict__ d64, const TV* __restrict__ X,
                              const double* __restrict__ kdiag_rows, const double* __restrict__ tau,
                              double* __restrict__ var_out, unsigned* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < n_cols; c += nw) {
    const int64_t r = r0 + c;
    double v;
    if (unit_rhs(tau, kdiag_rows, r)) {
      v = (1.0 - (double)X[r * R + c]) / tau[r];
    } else {
      double acc = 0;
      for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
        int32_t j = col[e];
        acc += d64[j] * (double)val[e] * (double)X[(int64_t)j * R + c];
      }
      acc = warp_sum(acc);
      v = kdiag_rows[r] - acc;
    }
    if (lane == 0) {
      if (!isfinite(v)) atomicOr(flags, kFlagNonFinite);
      var_out[r] = v;
    }
  }
}

// Query pairs interleaved as rows (2p, 2p + 1) of a query panel: the cross
// term v_{2p+1}^T B^-1 v_{2p} from the solution column of row 2p and the
// stored entries of row 2p + 1 (both rows sit in the same panel group).
template <typename TA, typename TV>
__global__ void k_panel_pair_cross(int64_t r0, int64_t n_cols, int R,
                                   const int64_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col, const TA* __restrict__ val,
                                   const double* __restrict__ d64, const TV* __restrict__ X,
                                   double* __restrict__ cross) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cn = 2 * warp; cn + 1 < n_cols; cn += 2 * nw) {
    const int64_t rf = r0 + cn + 1;  // far row; near column cn
    double acc = 0;
    for (int64_t e = row_ptr[rf] + lane; e < row_ptr[rf + 1]; e += 32) {
      const int32_t j = col[e];
      acc += d64[j] * (double)val[e] * (double)X[(int64_t)j * R + cn];
    }
    acc = warp_sum(acc);
    if (lane == 0) cross[(r0 + cn) / 2] = acc;
  }
}

// Groups of G consecutive rows (a sightline's points) in one panel group:
// cross[g * G (G - 1) / 2 + k] = v_b^T B^-1 v_a for the k-th pair a < b of
// group g (row-major over a), i.e. the far row's entries against the near
// column's solution.  Rows r0 .. r0 + n_cols - 1 are whole groups.
template <typename TA, typename TV>
__global__ void k_panel_group_cross(int64_t r0, int64_t n_cols, int R, int G,
                                    const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col, const TA* __restrict__ val,
                                    const double* __restrict__ d64, const TV* __restrict__ X,
                                    double* __restrict__ cross) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int npq = G * (G - 1) / 2;
  const int64_t ng = n_cols / G;
  for (int64_t t = warp; t < ng * npq; t += nw) {
    const int64_t gl = t / npq;
    int k = (int)(t - gl * npq), a = 0;
    while (k >= G - 1 - a) {
      k -= G - 1 - a;
      ++a;
    }
    const int b = a + 1 + k;
    const int64_t cn = gl * G + a;         // near column
    const int64_t rf = r0 + gl * G + b;    // far row
    double acc = 0;
    for (int64_t e = row_ptr[rf] + lane; e < row_ptr[rf + 1]; e += 32) {
      const int32_t j = col[e];
      acc += d64[j] * (double)val[e] * (double)X[(int64_t)j * R + cn];
    }
    acc = warp_sum(acc);
    if (lane == 0) cross[(r0 / G + gl) * npq + (t - gl * npq)] = acc;
  }
}

// Probed variances: star r reads its estimate from the column of its colour
// class (when that class is in this panel).
template <typename TA, typename TV>
__global__ void k_panel_final_probe(int64_t n, int64_t c0, int64_t n_cols, int R,
                                    const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col, const TA* __restrict__ val,
                                    const double* __restrict__ d64, const TV* __restrict__ X,
                                    const double* __restrict__ kdiag, const double* __restrict__ tau,
                                    const int32_t* __restrict__ pcol, double* __restrict__ var_out,
                                    unsigned* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    const int64_t k = (int64_t)pcol[r] - c0;
    if (k < 0 || k >= n_cols) continue;
    double v;
    if (unit_rhs(tau, kdiag, r)) {
      v = (1.0 - (double)X[r * R + k]) / tau[r];
    } else {
      double acc = 0;
      for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
        const int32_t j = col[e];
        acc += d64[j] * (double)val[e] * (double)X[(int64_t)j * R + k];
      }
      acc = warp_sum(acc);
      v = kdiag[r] - acc;
    }
    if (lane == 0) {
      if (!isfinite(v)) atomicOr(flags, kFlagNonFinite);
      var_out[r] = v;
    }
  }
}

// ---------------------------------------------------------------- host
static int vec_grid(gm_ctx* c) { return 2 * sm_count(c); }

template <typename TA, typename TV>
static gm_status cg_single(gm_ctx* c, const TV* rhs, TV* x, double tol, int max_it,
                           int64_t* iters, double* rel_resid) {
  Workspace& ws = W(c);
  const int64_t n = c->n;
  const int G = vec_grid(c);
  cudaStream_t st = c->stream;
  TV *r = (TV*)ws.r.p, *p = (TV*)ws.p.p, *pd = (TV*)ws.pd.p, *q = (TV*)ws.q.p;
  const TV *dv = (const TV*)ws.dv.p, *minv = (const TV*)ws.minv.p;
  double* part = (double*)ws.part.p;
  double* hp = (double*)c->h_pinned;
  if (((uintptr_t)c->col | (uintptr_t)c->val) & 15)
    return set_error(c, GM_E_INVAL, "CSR arrays must be 16-byte aligned");
  GM_PROF(c, "k_cg_init");
  k_cg_init<TV><<<G, kBT, 0, st>>>(n, rhs, minv, dv, x, r, p, pd, part);
  GM_LAUNCH_CHECK(c);
  // deflated preconditioner (FP32 contexts of one field, prepared this refresh)
  const bool defl = sizeof(TV) == 4 && c->cfg.deflate > 0 && c->n_fields == 1 && deflate_ready(c);
  if (defl) {
    gm_status ds = deflate1_rhs(c, (const float*)r, part + G);  // rz slot of iteration 1
    if (ds == GM_OK)
      ds = deflate1_update(c, (const float*)minv, (const float*)dv, nullptr, G, 0, 0,
                           (const float*)r, (float*)p, (float*)pd);
    if (ds != GM_OK) return ds;
  }
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hp, part + 4 * G, G * sizeof(double), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  double bb = 0;
  for (int k = 0; k < G; ++k) bb += hp[k];
  *iters = 0;
  *rel_resid = 0;
  if (!(bb > 0)) return GM_OK;
  const int check = 8;
  double rr = bb;
  int it = 1;
  for (; it <= max_it; ++it) {
    GM_PROF(c, "k_apply_B");
    k_apply_B<TA, TV><<<G, kBTB, 0, st>>>(n, c->row_ptr, c->col, (const TA*)c->val, dv, p, pd, q, part);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_cg_update1");
    k_cg_update1<TV><<<G, kBT, 0, st>>>(n, it, minv, x, r, p, q, part, c->d_flags);
    GM_LAUNCH_CHECK(c);
    if (it % check == 0 || it == max_it) {
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hp, part + 3 * G, G * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
      rr = 0;
      for (int k = 0; k < G; ++k) rr += hp[k];
      if (!std::isfinite(rr)) return set_error(c, GM_E_NONFINITE, "CG residual is not finite");
      if (rr <= tol * tol * bb) break;
    }
    if (defl) {
      const int prev = (it & 1) ? 1 : 2, next = (it & 1) ? 2 : 1;
      gm_status ds = deflate1_rhs(c, (const float*)r, part + next * G);
      if (ds == GM_OK)
        ds = deflate1_update(c, (const float*)minv, (const float*)dv, part, G, prev, next,
                             (const float*)r, (float*)p, (float*)pd);
      if (ds != GM_OK) return ds;
    } else {
      GM_PROF(c, "k_cg_update2");
      k_cg_update2<TV><<<G, kBT, 0, st>>>(n, it, minv, dv, r, p, pd, part);
      GM_LAUNCH_CHECK(c);
    }
  }
  *iters = std::min(it, max_it);
  *rel_resid = std::sqrt(rr / bb);
  return GM_OK;
}

static bool ensure_vecs(gm_ctx* c, size_t tv) {
  Workspace& ws = W(c);
  const size_t n = (size_t)c->n;
  const int G = vec_grid(c);
  bool ok = true;
  for (Buffer* b : {&ws.b64, &ws.w64, &ws.x64, &ws.r64, &ws.d64, &ws.minv64, &ws.dx64, &ws.kdx64})
    ok = ok && ensure(c, *b, n * sizeof(double));
  ok = ok && ensure(c, ws.r32, n * sizeof(float));
  for (Buffer* b : {&ws.x, &ws.r, &ws.p, &ws.pd, &ws.q, &ws.dv, &ws.minv})
    ok = ok && ensure(c, *b, n * tv);
  ok = ok && ensure(c, ws.part, 8 * (size_t)G * sizeof(double));
  return ok;
}

template <typename TA, typename TV>
static gm_status posterior_mean(gm_ctx* c, int64_t* iters, double* resid) {
  Workspace& ws = W(c);
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  const int eb = (int)std::min<int64_t>(ceil_div(n, 256), 8 * sms);
  const int wb = (int)std::min<int64_t>(ceil_div(n * 32, 256), 16 * sms);
  double *b64 = (double*)ws.b64.p, *w64 = (double*)ws.w64.p, *x64 = (double*)ws.x64.p,
         *r64 = (double*)ws.r64.p, *d64 = (double*)ws.d64.p;
  if (((uintptr_t)c->col | (uintptr_t)c->val) & 15)
    return set_error(c, GM_E_INVAL, "CSR arrays must be 16-byte aligned");
  // b = nu - tau m ; w = K b ; rhs = d o w
  GM_PROF(c, "k_site_rhs");
  k_site_rhs<<<eb, 256, 0, st>>>(n, c->nu, c->tau, c->prior_m, b64);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_spmv");
  k_spmv<TA, double><<<wb, 256, 0, st>>>(n, c->row_ptr, c->col, (const TA*)c->val, b64, nullptr, w64);
  GM_LAUNCH_CHECK(c);
  const double tol = c->cfg.cg_tol;
  const int max_it = c->cfg.cg_max_iter;
  gm_status s;
  if (sizeof(TV) == 8) {
    GM_PROF(c, "k_scale");
    k_scale<double><<<eb, 256, 0, st>>>(n, d64, w64, r64);  // rhs
    GM_LAUNCH_CHECK(c);
    s = cg_single<TA, double>(c, r64, x64, tol, max_it, iters, resid);
    if (s != GM_OK) return s;
    GM_PROF(c, "k_alpha");
    k_alpha<double><<<eb, 256, 0, st>>>(n, b64, d64, x64, c->alpha);
  } else {
    // FP32 CG on FP64-recomputed residuals (iterative refinement):
    // r = rhs - B x in FP64, solve B e = r in FP32, x += e, until ||r|| <= tol ||rhs||.
    double* rhs64 = w64;  // d o (K b), in place
    GM_PROF(c, "k_scale");
    k_scale<double><<<eb, 256, 0, st>>>(n, d64, w64, rhs64);
    GM_LAUNCH_CHECK(c);
    GM_CUDA_CHECK(c, cudaMemsetAsync(x64, 0, n * sizeof(double), st));
    float* r32 = (float*)ws.r32.p;
    float* e32 = (float*)ws.x.p;
    double* dx64 = (double*)ws.dx64.p;
    double* kdx64 = (double*)ws.kdx64.p;
    double* part = (double*)ws.part.p;
    double* hp = (double*)c->h_pinned;
    const int G = vec_grid(c);
    int64_t total = 0;
    double rel = 0;
    for (int outer = 0; outer < 20; ++outer) {
      GM_PROF(c, "k_scale");
      k_scale<double><<<eb, 256, 0, st>>>(n, d64, x64, dx64);
      GM_LAUNCH_CHECK(c);
      GM_PROF(c, "k_spmv");
      k_spmv<TA, double><<<wb, 256, 0, st>>>(n, c->row_ptr, c->col, (const TA*)c->val, dx64,
                                             nullptr, kdx64);
      GM_LAUNCH_CHECK(c);
      GM_PROF(c, "k_refine_resid");
      k_refine_resid<<<G, kBT, 0, st>>>(n, rhs64, x64, d64, kdx64, r64, r32, part + 6 * G);
      GM_LAUNCH_CHECK(c);
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hp, part + 6 * G, 2 * G * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
      double rr = 0, bb = 0;
      for (int k = 0; k < G; ++k) {
        rr += hp[k];
        bb += hp[G + k];
      }
      if (!std::isfinite(rr)) return set_error(c, GM_E_NONFINITE, "refined residual is not finite");
      rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
      if (rel <= tol) break;
      int64_t it = 0;
      double inner_rel = 0;
      // inner tolerance: enough to gain several digits per refinement step
      s = cg_single<TA, float>(c, r32, e32, std::max(1e-5, 0.1 * tol / rel), max_it, &it,
                               &inner_rel);
      if (s != GM_OK) return s;
      total += it;
      GM_PROF(c, "k_refine_add");
      k_refine_add<<<eb, 256, 0, st>>>(n, x64, e32, d64, dx64);
      GM_LAUNCH_CHECK(c);
    }
    *iters = total;
    *resid = rel;
    GM_PROF(c, "k_alpha");
    k_alpha<double><<<eb, 256, 0, st>>>(n, b64, d64, x64, c->alpha);
  }
  GM_LAUNCH_CHECK(c);
  // mu = m + K alpha
  GM_PROF(c, "k_spmv");
  k_spmv<TA, double><<<wb, 256, 0, st>>>(n, c->row_ptr, c->col, (const TA*)c->val, c->alpha,
                                         c->prior_m, c->mu);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

// Panel product Q = P + d o (K PD) with the tiled kernel when available.
// *nbx_used: rows of per-column partials written to pa (the reduction's nbx).
template <typename TA, typename TV>
static gm_status panel_product(gm_ctx* c, int64_t n, int64_t R, int nbx, dim3 grid, const TV* dv,
                               const TV* P, const TV* PD, TV* Q, double* pa, int* nbx_used,
                               bool planes_ready = false) {
  *nbx_used = nbx;
  if (sizeof(TV) == 4 && c->tc_nblk > 0) {
    *nbx_used = (int)c->tc_nblk;
    return panel_spmm_tc(c, n, (int)R, (const float*)dv, (const float*)P, (const float*)PD,
                         (float*)Q, pa, planes_ready);
  }
  if (sizeof(TV) == 4 && c->t_nblk > 0)
    return panel_spmm_tiled(c, n, (int)R, nbx, (const float*)dv, (const float*)P,
                            (const float*)PD, (float*)Q, pa);
  GM_PROF(c, "k_panel_spmm");
  k_panel_spmm<TA, TV><<<grid, kBT, 0, c->stream>>>(n, (int)R, c->row_ptr, c->col,
                                                    (const TA*)c->val, dv, P, PD, Q, pa);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status panel_apply_B_f32(gm_ctx* c, int R, const float* dv, const float* P, const float* PD,
                            float* Q, double* part) {
  const int sms = sm_count(c);
  const int nbx = std::max(1, (int)std::min<int64_t>(ceil_div(c->n, 8),
                                                     (int64_t)(4 * sms * 32 / (R / 32 + 1)) + 1));
  dim3 grid(nbx, (unsigned)(R / 32));
  int nbu = nbx;
  return panel_product<float, float>(c, c->n, R, nbx, grid, dv, P, PD, Q, part, &nbu);
}

// stars: the rows are the stars themselves (unit right-hand sides allowed,
// and the solutions may seed the next call: warm start when the previous
// call solved the stars in one panel of the same width).
template <typename TA, typename TV>
static gm_status panels(gm_ctx* c, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                        const void* val, const double* kdiag_rows, double* var_out,
                        int64_t* iters_out, double* resid_out, bool stars,
                        double* pair_cross = nullptr, int cross_group = 2) {
  const bool warm = stars;
  // probed variances: one column per colour class instead of one per star
  const bool probe = stars && c->probe_colour && c->probe_factor_done > 0 && c->n_fields == 1;
  const int64_t n_cols_all = probe ? (int64_t)c->h_probe_ncol[0] : n_rows;
  Workspace& ws = W(c);
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  // panel width: all rows if they fit a memory budget, in multiples of 32
  int64_t R = c->cfg.rhs_panel > 0 ? c->cfg.rhs_panel : 0;
  if (R == 0) {
    size_t free_b = 0, tot_b = 0;
    cudaMemGetInfo(&free_b, &tot_b);
    // five panel arrays (+ three BF16 planes of PD for the tensor-core
    // product) within half of the free memory plus what this context's panel
    // arrays already hold (they are reused or replaced), at most 160 GB: the
    // width then stays the same from one refresh to the next
    const size_t held = ws.P_X.bytes + ws.P_R.bytes + ws.P_P.bytes + ws.P_PD.bytes +
                        ws.P_Q.bytes + (sizeof(TV) == 4 ? c->tc_planes.bytes : 0);
    double budget = std::min<double>(0.5 * ((double)free_b + (double)held), 160e9);
    const double per = 5.0 * sizeof(TV) + (sizeof(TV) == 4 && c->tc_nblk > 0 ? 6.0 : 0.0);
    R = (int64_t)(budget / (per * (double)n));
  }
  R = std::max<int64_t>(32, std::min<int64_t>(R, ceil_div(n_cols_all, 32) * 32));
  R = (R / 32) * 32;
  c->stats.variance_panel_width = R;
  const int nbx = std::max(1, (int)std::min<int64_t>(ceil_div(n, 8), (int64_t)(4 * sms * 32 / (R / 32 + 1)) + 1));
  const size_t pbytes = (size_t)n * R * sizeof(TV);
  // spectral deflation of the preconditioner (FP32 star panels of one field;
  // the vectors are prepared per refresh, before the mean solve), in its
  // tensor-core form when the context has tensor-core tiles
  const bool defl =
      stars && sizeof(TV) == 4 && c->cfg.deflate > 0 && c->n_fields == 1 && deflate_ready(c);
  const bool defl_tc = defl && deflate_tc(c);
  const int nch = defl_tc ? deflate_tc_chunks(c, (int)R) : 0;  // partial rows of its step
  // partial rows: the panel product may write more rows (one per 128-row
  // tile), the tensor-core deflation step one per row chunk; then the rows
  // of the deflation term of r^T z (1, or 8 in the tensor-core form)
  const int64_t rows_a = std::max<int64_t>(std::max<int64_t>(nbx, nch),
                                           sizeof(TV) == 4 ? c->tc_nblk : 0);
  const int64_t rows_b = std::max<int64_t>(nbx, nch);
  const int ncorr = defl ? (defl_tc ? 8 : 1) : 0;
  bool ok = ensure(c, ws.P_X, pbytes) && ensure(c, ws.P_R, pbytes) && ensure(c, ws.P_P, pbytes) &&
            ensure(c, ws.P_PD, pbytes) && ensure(c, ws.P_Q, pbytes) &&
            ensure(c, ws.P_part, (size_t)(rows_a + rows_b + std::max(ncorr, 1)) * R *
                                     sizeof(double)) &&
            ensure(c, ws.P_scal, 6 * (size_t)R * sizeof(double)) &&
            ensure(c, ws.P_active, (size_t)(R + 32) * sizeof(int));
  if (!ok) return set_error(c, GM_E_NOMEM, "variance panels");
  TV *X = (TV*)ws.P_X.p, *Rr = (TV*)ws.P_R.p, *P = (TV*)ws.P_P.p, *PD = (TV*)ws.P_PD.p,
     *Q = (TV*)ws.P_Q.p;
  double* pa = (double*)ws.P_part.p;
  double* pb = pa + (size_t)rows_a * R;
  double* corr = pb + (size_t)rows_b * R;  // the deflation rows of r^T z
  double* scal = (double*)ws.P_scal.p;
  int* active = (int*)ws.P_active.p;
  int* n_active = active + R;
  const TV *dv = (const TV*)ws.dv.p, *minv = (const TV*)ws.minv.p;
  // FP32 panels stop at the FP32 rounding floor of the relative residual
  const double tol = sizeof(TV) == 4 ? std::max(c->cfg.cg_tol, 1e-5) : c->cfg.cg_tol;
  const double tol2 = tol * tol;
  const int max_it = c->cfg.cg_max_iter;
  int* hn = (int*)c->h_pinned;
  dim3 grid(nbx, (unsigned)(R / 32));
  const int rb = (int)std::min<int64_t>(ceil_div(n_rows * 32, 256), 16 * sms);
  const int redb = (int)ceil_div(R, 256);
  int64_t total_it = 0;
  const int tb = (int)std::min<int64_t>(ceil_div(n, 256), 16 * sms);
  for (int64_t r0 = 0; r0 < n_cols_all; r0 += R) {
    const int64_t ncols = std::min<int64_t>(R, n_cols_all - r0);
    GM_CUDA_CHECK(c, cudaMemsetAsync(Rr, 0, pbytes, st));
    if (probe && c->probe_factor_done >= 2.0) {
      GM_PROF(c, "k_panel_rhs_probe");
      k_panel_rhs_probe_w<TA, TV><<<(int)std::min<int64_t>(ceil_div(n * 32, 256), 16 * sms), 256,
                                    0, st>>>(n, r0, ncols, (int)R, row_ptr, col, (const TA*)val,
                                             dv, c->tau, kdiag_rows, c->probe_colour, Rr);
    } else if (probe) {
      GM_PROF(c, "k_panel_rhs_probe");
      k_panel_rhs_probe<TA, TV><<<tb, 256, 0, st>>>(n, r0, ncols, (int)R, row_ptr, col,
                                                    (const TA*)val, dv, c->tau, kdiag_rows,
                                                    c->probe_colour, Rr);
    } else {
      GM_PROF(c, "k_panel_rhs");
      k_panel_rhs<TA, TV><<<rb, 256, 0, st>>>(r0, ncols, (int)R, row_ptr, col, (const TA*)val, dv,
                                              warm ? c->tau : nullptr, kdiag_rows, Rr);
    }
    GM_LAUNCH_CHECK(c);
    const bool use_warm = warm && c->cfg.warm_start && c->warm_R == R && n_cols_all <= R &&
                          c->warm_probe == (probe ? 1 : 0);
    if (use_warm) {
      GM_PROF(c, "k_panel_scale");
      k_panel_scale<TV><<<grid, kBT, 0, st>>>(n, (int)R, dv, X, PD);
      GM_LAUNCH_CHECK(c);
      int nbu = nbx;
      gm_status ss = panel_product<TA, TV>(c, n, R, nbx, grid, dv, X, PD, Q, pa, &nbu);
      if (ss != GM_OK) return ss;
      GM_PROF(c, "k_panel_init_warm");
      k_panel_init_warm<TV><<<grid, kBT, 0, st>>>(n, (int)R, minv, dv, Rr, Q, P, PD, pa, pb);
      GM_LAUNCH_CHECK(c);
    } else {
      GM_PROF(c, "k_panel_init");
      k_panel_init<TV><<<grid, kBT, 0, st>>>(n, (int)R, minv, dv, X, Rr, P, PD, pa, pb);
      GM_LAUNCH_CHECK(c);
    }
    // the BF16 planes of PD were written by the deflation update (the
    // asynchronous tile product then skips its split)
    bool planes = false;
    if (defl) {
      // z = M_d^-1 r for the initial residuals: P, PD and the rz rows
      gm_status ds;
      if (defl_tc) {
        planes = tc_variant(c, (int)R) == 4;
        ds = deflate_step_tc(c, (int)R, nch, nullptr, (const float*)minv, (float*)X, (float*)Rr,
                             (const float*)P, (const float*)Q, nullptr, nullptr, corr);
        if (ds == GM_OK)
          ds = deflate_update_tc(c, (int)R, (const float*)minv, (const float*)dv, nullptr,
                                 nullptr, (const float*)Rr, (float*)P, (float*)PD, planes);
      } else {
        ds = deflate_rhs(c, (int)R, (const float*)Rr, corr);
        if (ds == GM_OK)
          ds = deflate_update(c, (int)R, nbx, (const float*)minv, (const float*)dv, nullptr,
                              nullptr, (const float*)Rr, (float*)P, (float*)PD);
      }
      if (ds != GM_OK) return ds;
    }
    GM_CUDA_CHECK(c, cudaMemsetAsync(n_active, 0, sizeof(int), st));
    GM_PROF(c, "k_panel_reduce");
    k_panel_reduce<<<redb, 256, 0, st>>>(0, nbx, (int)R, ncols, tol2, 0, max_it, pa, pb, corr,
                                         ncorr, scal, active, n_active, c->d_flags);
    GM_LAUNCH_CHECK(c);
    const int check = 8;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(hn, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
    int it = *hn == 0 ? 0 : 1;  // no active column (all right-hand sides zero): no iteration
    for (; it >= 1 && it <= max_it; ++it) {
      int nbu = nbx;
      {
        gm_status ss = panel_product<TA, TV>(c, n, R, nbx, grid, dv, P, PD, Q, pa, &nbu, planes);
        if (ss != GM_OK) return ss;
      }
      GM_PROF(c, "k_panel_reduce");
      k_panel_reduce<<<redb, 256, 0, st>>>(1, nbu, (int)R, ncols, tol2, it, max_it, pa, nullptr,
                                           nullptr, 0, scal, active, n_active, c->d_flags);
      GM_LAUNCH_CHECK(c);
      int nbr = nbx;  // partial rows of rz / rr
      if (defl_tc) {
        // X, Rr update fused with C = Y^T Rr and the deflation rows
        gm_status ds = deflate_step_tc(c, (int)R, nch, scal, (const float*)minv, (float*)X,
                                       (float*)Rr, (const float*)P, (const float*)Q, pa, pb, corr);
        if (ds != GM_OK) return ds;
        nbr = nch;
      } else {
        GM_PROF(c, "k_panel_update1");
        k_panel_update1<TV><<<grid, kBT, 0, st>>>(n, (int)R, minv, scal, X, Rr, P, Q, pa, pb);
        GM_LAUNCH_CHECK(c);
        if (defl) {
          gm_status ds = deflate_rhs(c, (int)R, (const float*)Rr, corr);
          if (ds != GM_OK) return ds;
        }
      }
      GM_CUDA_CHECK(c, cudaMemsetAsync(n_active, 0, sizeof(int), st));
      GM_PROF(c, "k_panel_reduce");
      k_panel_reduce<<<redb, 256, 0, st>>>(2, nbr, (int)R, ncols, tol2, it, max_it, pa, pb, corr,
                                           ncorr, scal, active, n_active, c->d_flags);
      GM_LAUNCH_CHECK(c);
      planes = false;
      if (defl_tc) {
        planes = tc_variant(c, (int)R) == 4;
        gm_status ds = deflate_update_tc(c, (int)R, (const float*)minv, (const float*)dv,
                                         scal + R, active, (const float*)Rr, (float*)P,
                                         (float*)PD, planes);
        if (ds != GM_OK) return ds;
      } else if (defl) {
        gm_status ds = deflate_update(c, (int)R, nbx, (const float*)minv, (const float*)dv,
                                      scal + R, active, (const float*)Rr, (float*)P, (float*)PD);
        if (ds != GM_OK) return ds;
      } else {
        GM_PROF(c, "k_panel_update2");
        k_panel_update2<TV><<<grid, kBT, 0, st>>>(n, (int)R, minv, dv, scal, active, Rr, P, PD);
        GM_LAUNCH_CHECK(c);
      }
      if (it % check == 0 || it == max_it) {
        GM_CUDA_CHECK(c, cudaMemcpyAsync(hn, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
        if (*hn == 0) break;
      }
    }
    total_it += std::min(it, max_it);
    if (probe) {
      GM_PROF(c, "k_panel_final_probe");
      k_panel_final_probe<TA, TV><<<(int)std::min<int64_t>(ceil_div(n * 32, 256), 16 * sms), 256,
                                    0, st>>>(n, r0, ncols, (int)R, row_ptr, col, (const TA*)val,
                                             (const double*)ws.d64.p, X, kdiag_rows, c->tau,
                                             c->probe_colour, var_out, c->d_flags);
    } else {
      GM_PROF(c, "k_panel_final");
      k_panel_final<TA, TV><<<rb, 256, 0, st>>>(r0, ncols, (int)R, row_ptr, col, (const TA*)val,
                                                (const double*)ws.d64.p, X, kdiag_rows,
                                                warm ? c->tau : nullptr, var_out, c->d_flags);
    }
    GM_LAUNCH_CHECK(c);
    if (pair_cross && !probe && cross_group > 2) {  // G divides R: groups share the panel
      GM_PROF(c, "k_panel_group_cross");
      k_panel_group_cross<TA, TV><<<rb, 256, 0, st>>>(r0, ncols, (int)R, cross_group, row_ptr,
                                                      col, (const TA*)val,
                                                      (const double*)ws.d64.p, X, pair_cross);
      GM_LAUNCH_CHECK(c);
    } else if (pair_cross && !probe) {  // R is even: a pair's rows share the group
      GM_PROF(c, "k_panel_pair_cross");
      k_panel_pair_cross<TA, TV><<<rb, 256, 0, st>>>(r0, ncols, (int)R, row_ptr, col,
                                                     (const TA*)val, (const double*)ws.d64.p, X,
                                                     pair_cross);
      GM_LAUNCH_CHECK(c);
    }
  }
  // worst relative residual over the last panel's columns
  std::vector<double> h(2 * R);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), scal + 4 * R, 2 * R * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  double worst = 0;
  for (int64_t k = 0; k < R; ++k)
    if (h[k] > 0) worst = std::max(worst, std::sqrt(h[R + k] / h[k]));
  *iters_out = total_it;
  *resid_out = worst;
  c->warm_R = (warm && n_cols_all <= R) ? R : 0;
  c->warm_probe = probe ? 1 : 0;
  return GM_OK;
}

static gm_status prepare_precond(gm_ctx* c) {
  const bool f32 = c->cfg.precision == GM_PREC_FP32;
  if (!ensure_vecs(c, f32 ? sizeof(float) : sizeof(double)))
    return set_error(c, GM_E_NOMEM, "CG vectors");
  Workspace& ws = W(c);
  const int eb = (int)std::min<int64_t>(ceil_div(c->n, 256), 8 * sm_count(c));
  GM_PROF(c, "k_precond");
  if (f32)
    k_precond<float><<<eb, 256, 0, c->stream>>>(c->n, c->tau, c->kdiag, (float*)ws.dv.p,
                                                (float*)ws.minv.p, (double*)ws.d64.p,
                                                (double*)ws.minv64.p);
  else
    k_precond<double><<<eb, 256, 0, c->stream>>>(c->n, c->tau, c->kdiag, (double*)ws.dv.p,
                                                 (double*)ws.minv.p, (double*)ws.d64.p,
                                                 (double*)ws.minv64.p);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status refresh_posterior(gm_ctx* c) {
  gm_status s = prepare_precond(c);
  if (s != GM_OK) return s;
  int64_t it_m = 0, it_v = 0;
  double res_m = 0, res_v = 0;
  if (c->cfg.precision == GM_PREC_FP32) {
    // deflation vectors for this refresh (mean CG and variance panels)
    if (c->cfg.deflate > 0 && c->n_fields == 1) {
      s = deflate_prepare(c, (const float*)W(c).dv.p, (const float*)W(c).minv.p);
      if (s != GM_OK) return s;
    }
    s = posterior_mean<float, float>(c, &it_m, &res_m);
    if (s == GM_OK && c->n_fields > 1)
      s = panels_fields(c, (const float*)W(c).dv.p, (const float*)W(c).minv.p,
                        (const double*)W(c).d64.p, c->var, &it_v, &res_v);
    else if (s == GM_OK)
      s = panels<float, float>(c, c->n, c->row_ptr, c->col, c->val, c->kdiag, c->var, &it_v, &res_v,
                               true);
  } else {
    s = posterior_mean<double, double>(c, &it_m, &res_m);
    if (s == GM_OK)
      s = panels<double, double>(c, c->n, c->row_ptr, c->col, c->val, c->kdiag, c->var, &it_v,
                                 &res_v, true);
  }
  if (s != GM_OK) return s;
  c->stats.cg_iters_mean = it_m;
  c->stats.cg_iters_var = it_v;
  c->stats.cg_resid_mean = res_m;
  c->stats.cg_resid_var = res_v;
  c->post_valid = true;
  return GM_OK;
}

gm_status posterior_mean_only(gm_ctx* c) {
  gm_status s = prepare_precond(c);
  if (s != GM_OK) return s;
  int64_t it = 0;
  double res = 0;
  if (c->cfg.precision == GM_PREC_FP32) {
    if (c->cfg.deflate > 0 && c->n_fields == 1) {
      s = deflate_prepare(c, (const float*)W(c).dv.p, (const float*)W(c).minv.p);
      if (s != GM_OK) return s;
    }
    s = posterior_mean<float, float>(c, &it, &res);
  } else {
    s = posterior_mean<double, double>(c, &it, &res);
  }
  if (s != GM_OK) return s;
  c->stats.cg_iters_mean = it;
  c->stats.cg_resid_mean = res;
  return GM_OK;
}

gm_status panel_variances(gm_ctx* c, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                          const void* val, const double* kdiag_rows, double* var_out,
                          int64_t* iters_out, double* resid_out, double* pair_cross,
                          int cross_group) {
  gm_status s = prepare_precond(c);
  if (s != GM_OK) return s;
  if (c->cfg.precision == GM_PREC_FP32)
    return panels<float, float>(c, n_rows, row_ptr, col, val, kdiag_rows, var_out, iters_out,
                                resid_out, false, pair_cross, cross_group);
  return panels<double, double>(c, n_rows, row_ptr, col, val, kdiag_rows, var_out, iters_out,
                                resid_out, false, pair_cross, cross_group);
}

gm_status csr_dot_alpha(gm_ctx* c, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                        const void* val, const double* alpha, const double* base, double* out) {
  const int wb = (int)std::min<int64_t>(ceil_div(n_rows * 32, 256), 16 * sm_count(c));
  if (n_rows == 0) return GM_OK;
  if (((uintptr_t)col | (uintptr_t)val) & 15)
    return set_error(c, GM_E_INVAL, "CSR arrays must be 16-byte aligned");
  GM_PROF(c, "k_spmv");
  if (c->cfg.precision == GM_PREC_FP32)
    k_spmv<float, double><<<wb, 256, 0, c->stream>>>(n_rows, row_ptr, col, (const float*)val, alpha, base, out);
  else
    k_spmv<double, double><<<wb, 256, 0, c->stream>>>(n_rows, row_ptr, col, (const double*)val, alpha, base, out);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm
