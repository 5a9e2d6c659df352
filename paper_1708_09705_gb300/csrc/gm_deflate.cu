// Spectral deflation of the variance-panel preconditioner.
//
// The panel CG solves B X = V with the Jacobi preconditioner M^-1 = diag(B)^-1.
// The spectrum of the scaled operator B~ = M^-1/2 B M^-1/2 has a long tail of
// large eigenvalues (sightlines crowded along the line of sight), which
// costs Jacobi-PCG most of its iterations.  Given k orthonormal approximate
// eigenvectors V of B~ with Ritz values theta (exact Rayleigh-Ritz values on
// span V), Y = M^-1/2 V is M-orthonormal and
//     M_d^-1 = M^-1 + Y (Theta^-1 - I) Y^T
// is symmetric positive definite (in the M^1/2 frame it is I + V (Theta^-1 - I)
// V^T, with eigenvalues 1 and 1/theta > 0), and maps the Ritz directions of
// M^-1 B to eigenvalue ~1: the "spectral preconditioner" of deflated Krylov
// methods (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Sect.
// 9.6; Carpentieri, Duff & Giraud 2003).  The CG is unchanged apart from
// applying M_d^-1 to the residuals: z = M^-1 r + Yw (Y^T r), Yw = Y (Theta^-1 - I),
// and r^T z = r^T M^-1 r + sum_j w_j (Y^T r)_j^2.
//
// V is obtained per posterior refresh by a few steps of orthogonal subspace
// iteration on B~ (each: one panel product of k columns and two Cholesky-QR
// passes with FP64 Gram matrices), warm-started from the previous refresh,
// followed by Rayleigh-Ritz (FP64 Jacobi eigen-solver on the host).
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kDefK = 64;          // deflation vectors
constexpr int kDefIters = 8;       // subspace-iteration steps, first refresh
constexpr int kDefItersWarm = 3;   // ... later refreshes (warm start)
constexpr int kDefRows = 256;      // rows per block of the Y^T R kernel

struct Deflation {
  int64_t n = 0;
  bool have_v = false;
  Buffer V, W, Y, Yw;              // n x k FP32 (row-major)
  Buffer P, PD, Q;                 // n x k panel product buffers
  Buffer part;                     // panel-product partials
  Buffer G, Gp;                    // k x k FP64 Gram / projection, partials per 64 rows
  Buffer Mk;                       // k x k FP32 matrix applied on the right
  Buffer ms;                       // n: M^-1/2
  Buffer Cp, C;                    // Y^T R: partials per row block, and the sum (k x R)
  Buffer wv;                       // k weights 1/theta - 1 (FP32)
  Buffer cpart1, c1;               // single right-hand side: Y^T r partials and sum
  Buffer yimg, ywimg, cimg, Cp2;   // tensor-core form: images of Y^T, Yw, C^T; C partials
  std::vector<double> theta;       // Ritz values of this refresh
  bool ready = false;              // Y, Yw, wv valid for this refresh
  bool tc = false;                 // ... and the images of Y^T and Yw
};

static Deflation& D(gm_ctx* c) {
  if (!c->defl) c->defl = new Deflation();
  return *c->defl;
}

void deflate_free(gm_ctx* c) {
  delete c->defl;
  c->defl = nullptr;
}

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ uint64_t df_mix(uint64_t x) {  // SplitMix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// deterministic start block: entries uniform in [-1/2, 1/2)
__global__ void k_df_init(int64_t n, float* __restrict__ V) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kDefK;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = (float)((double)(df_mix((uint64_t)e) >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// P = ms o V, PD = d o P
__global__ void k_df_scale_in(int64_t n, const float* __restrict__ ms, const float* __restrict__ dv,
                              const float* __restrict__ V, float* __restrict__ P,
                              float* __restrict__ PD) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kDefK;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kDefK;
    const float p = ms[i] * V[e];
    P[e] = p;
    PD[e] = dv[i] * p;
  }
}

// W = ms o Q
__global__ void k_df_scale_out(int64_t n, const float* __restrict__ ms, const float* __restrict__ Q,
                               float* __restrict__ W) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kDefK;
       e += (int64_t)gridDim.x * blockDim.x)
    W[e] = ms[e / kDefK] * Q[e];
}

// Gp[rb][a][b] = sum over 64-row block rb of X[i][a] Z[i][b]; thread tile 16
// entries; the 64 x 64 row blocks of X and Z staged in shared memory.  The
// products of FP32 inputs are summed over the block's 64 rows in FP32 (about
// 64 roundings, ~1e-6 relative at worst: well inside what Cholesky-QR run
// twice and the Rayleigh-Ritz values need) and over blocks in FP64 (GB300's
// FP64 pipe, not the data, bounded the all-FP64 form).
__global__ void __launch_bounds__(256) k_df_gram(int64_t n, const float* __restrict__ X,
                                                 const float* __restrict__ Z,
                                                 double* __restrict__ Gp) {
  __shared__ float xs[64][kDefK], zs[64][kDefK];
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  for (int e = t; e < 64 * kDefK; e += 256) {
    const int r = e / kDefK, k = e - r * kDefK;
    const bool in = r0 + r < n;
    xs[r][k] = in ? X[(r0 + r) * kDefK + k] : 0.f;
    zs[r][k] = in ? Z[(r0 + r) * kDefK + k] : 0.f;
  }
  __syncthreads();
  const int a = t >> 2, b0 = 16 * (t & 3);
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int r = 0; r < 64; ++r) {
    const float xa = xs[r][a];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fmaf(xa, zs[r][b0 + q], acc[q]);
  }
  double* out = Gp + (int64_t)blockIdx.x * kDefK * kDefK + a * kDefK + b0;
#pragma unroll
  for (int q = 0; q < 16; ++q) out[q] = (double)acc[q];
}

// G = sum over row blocks of Gp (fixed order)
__global__ void k_df_gram_sum(int nb, const double* __restrict__ Gp, double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kDefK * kDefK) return;
  double s = 0.0;
  for (int q = 0; q < nb; ++q) s += Gp[(int64_t)q * kDefK * kDefK + e];
  G[e] = s;
}

// Out[i][:] = In[i][:] * M (k x k, row-major), row per thread group
__global__ void k_df_right(int64_t n, const float* __restrict__ In, const float* __restrict__ M,
                           float* __restrict__ Out) {
  __shared__ float sm[kDefK * kDefK];
  for (int e = threadIdx.x; e < kDefK * kDefK; e += blockDim.x) sm[e] = M[e];
  __syncthreads();
  // thread per (row, output column)
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kDefK;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kDefK;
    const int b = (int)(e - i * kDefK);
    const float* row = In + i * kDefK;
    float s = 0.f;
#pragma unroll 16
    for (int a = 0; a < kDefK; ++a) s = fmaf(row[a], sm[a * kDefK + b], s);
    Out[e] = s;
  }
}

// Y = ms o V, Yw = Y diag(w)
__global__ void k_df_make_y(int64_t n, const float* __restrict__ ms, const float* __restrict__ V,
                            const float* __restrict__ w, float* __restrict__ Y,
                            float* __restrict__ Yw) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kDefK;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kDefK;
    const int j = (int)(e - i * kDefK);
    const float y = ms[i] * V[e];
    Y[e] = y;
    Yw[e] = y * w[j];
  }
}

__global__ void k_df_ms(int64_t n, const float* __restrict__ minv, float* __restrict__ ms) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    ms[i] = sqrtf(minv[i]);
}

// Cp[rb][j][c] = sum over the block's rows i of Y[i][j] R[i][c] (split over
// row blocks of kDefRows).  Block tile: all 64 j x 128 columns; thread tile
// 4 j x 8 columns (register outer products), rows staged 32 at a time.
__global__ void __launch_bounds__(256) k_df_yt_r(int64_t n, int R, const float* __restrict__ Y,
                                                 const float* __restrict__ Rr,
                                                 float* __restrict__ Cp) {
  __shared__ __align__(16) float ys[32][kDefK];
  __shared__ __align__(16) float rs[32][128];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int c0 = blockIdx.x * 128;
  const int64_t rb = blockIdx.y;
  const int64_t i0 = rb * kDefRows, i1 = min(i0 + kDefRows, n);
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    const int cnt = (int)min((int64_t)32, i1 - ib);
    __syncthreads();
    for (int e = t; e < 32 * kDefK / 4; e += 256) {  // Y rows, float4
      const int r = e / (kDefK / 4), q = e - r * (kDefK / 4);
      reinterpret_cast<float4*>(ys[r])[q] =
          r < cnt ? *reinterpret_cast<const float4*>(Y + (ib + r) * kDefK + 4 * q)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int e = t; e < 32 * 32; e += 256) {  // R rows, 128 columns as float4
      const int r = e >> 5, q = e & 31;
      const int cc = c0 + 4 * q;
      reinterpret_cast<float4*>(rs[r])[q] =
          (r < cnt && cc < R) ? *reinterpret_cast<const float4*>(Rr + (ib + r) * R + cc)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    for (int r = 0; r < cnt; ++r) {
      const float4 a = reinterpret_cast<const float4*>(ys[r])[ty];
      const float4 b0 = reinterpret_cast<const float4*>(rs[r])[2 * tx];
      const float4 b1 = reinterpret_cast<const float4*>(rs[r])[2 * tx + 1];
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = 4 * ty + u;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int cc = c0 + 8 * tx + v;
      if (cc < R) Cp[(rb * kDefK + j) * R + cc] = acc[u][v];
    }
  }
}

// C[j][c] = sum_rb Cp[rb][j][c] in row-block order; thread per (j, c)
__global__ void k_df_sum(int R, int nrb, const float* __restrict__ Cp, float* __restrict__ C) {
  const int64_t tot = (int64_t)kDefK * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int rb = 0; rb < nrb; ++rb) s += Cp[(int64_t)rb * tot + e];
    C[e] = s;
  }
}

// corr[c] = sum_j w_j C[j][c]^2 (FP64), thread per column
__global__ void k_df_corr(int R, const float* __restrict__ C, const float* __restrict__ w,
                          double* __restrict__ corr) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    double cs = 0.0;
    for (int j = 0; j < kDefK; ++j) {
      const double v = C[(int64_t)j * R + c];
      cs += (double)w[j] * v * v;
    }
    corr[c] = cs;
  }
}

// P = M^-1 R + Yw C + beta P on active columns (all, beta 0, when active is
// null), PD = d o P.  Block tile 64 rows x 128 columns with Yw (transposed)
// and C staged in shared memory; thread tile 4 rows x 8 columns.
__global__ void __launch_bounds__(256) k_df_update(int64_t n, int R, const float* __restrict__ minv,
                                                   const float* __restrict__ dv,
                                                   const double* __restrict__ beta,
                                                   const int* __restrict__ active,
                                                   const float* __restrict__ Rr,
                                                   const float* __restrict__ Yw,
                                                   const float* __restrict__ C,
                                                   float* __restrict__ P, float* __restrict__ PD) {
  extern __shared__ __align__(16) float dsm[];
  float* ywt = dsm;                  // [64 k][64 rows]
  float* cs = dsm + kDefK * 64;      // [64 k][128 columns]
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int c0 = blockIdx.x * 128;
  const int64_t r0 = (int64_t)blockIdx.y * 64;
  for (int e = t; e < 64 * kDefK; e += 256) {  // Yw rows r0.., transposed
    const int r = e / kDefK, k = e - r * kDefK;
    ywt[k * 64 + r] = r0 + r < n ? Yw[(r0 + r) * kDefK + k] : 0.f;
  }
  for (int e = t; e < kDefK * 32; e += 256) {  // C, 128 columns as float4
    const int k = e >> 5, q = e & 31;
    const int cc = c0 + 4 * q;
    reinterpret_cast<float4*>(cs + k * 128)[q] =
        cc < R ? *reinterpret_cast<const float4*>(C + (int64_t)k * R + cc)
               : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 4
  for (int k = 0; k < kDefK; ++k) {
    const float4 a = reinterpret_cast<const float4*>(ywt + k * 64)[ty];
    const float4 b0 = reinterpret_cast<const float4*>(cs + k * 128)[2 * tx];
    const float4 b1 = reinterpret_cast<const float4*>(cs + k * 128)[2 * tx + 1];
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
  }
  const int cb = c0 + 8 * tx;
  if (cb >= R) return;
  bool act[8];
  float be[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    act[v] = active ? active[cb + v] != 0 : true;
    be[v] = (beta && act[v]) ? (float)beta[cb + v] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = r0 + 4 * ty + u;
    if (i >= n) break;
    const float m = minv[i], d = dv[i];
    const int64_t k0 = i * R + cb;
    float rv[8], pv[8], dd[8];
    *reinterpret_cast<float4*>(rv) = *reinterpret_cast<const float4*>(Rr + k0);
    *reinterpret_cast<float4*>(rv + 4) = *reinterpret_cast<const float4*>(Rr + k0 + 4);
    *reinterpret_cast<float4*>(pv) = *reinterpret_cast<const float4*>(P + k0);
    *reinterpret_cast<float4*>(pv + 4) = *reinterpret_cast<const float4*>(P + k0 + 4);
    *reinterpret_cast<float4*>(dd) = *reinterpret_cast<const float4*>(PD + k0);
    *reinterpret_cast<float4*>(dd + 4) = *reinterpret_cast<const float4*>(PD + k0 + 4);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if (act[v]) {  // frozen columns keep P and PD
        const float p = m * rv[v] + acc[u][v] + be[v] * pv[v];
        pv[v] = p;
        dd[v] = d * p;
      }
    }
    *reinterpret_cast<float4*>(P + k0) = *reinterpret_cast<const float4*>(pv);
    *reinterpret_cast<float4*>(P + k0 + 4) = *reinterpret_cast<const float4*>(pv + 4);
    *reinterpret_cast<float4*>(PD + k0) = *reinterpret_cast<const float4*>(dd);
    *reinterpret_cast<float4*>(PD + k0 + 4) = *reinterpret_cast<const float4*>(dd + 4);
  }
}

// ---- single right-hand side (the posterior-mean CG)
// cpart[b][j] = sum over block b's rows of Y[i][j] r[i] (FP64); warp per row
// (lanes j and j + 32), block partials summed over its warps in order.
__global__ void __launch_bounds__(256) k_df1_part(int64_t n, const float* __restrict__ Y,
                                                  const float* __restrict__ r,
                                                  double* __restrict__ cpart) {
  __shared__ double sh[8][kDefK];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += (int64_t)gridDim.x * 8) {
    const double ri = r[i];
    a0 += (double)Y[i * kDefK + lane] * ri;
    a1 += (double)Y[i * kDefK + 32 + lane] * ri;
  }
  sh[wib][lane] = a0;
  sh[wib][32 + lane] = a1;
  __syncthreads();
  if (threadIdx.x < kDefK) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w][threadIdx.x];
    cpart[(int64_t)blockIdx.x * kDefK + threadIdx.x] = s;
  }
}

// c = sum_b cpart[b] (in order); rz_slot[0] += sum_j w_j c_j^2.  One block of
// 64 threads.
// (Four threads per j sum every fourth partial row, then j's thread adds the
// four in order: the same fixed order on every call.)
__global__ void k_df1_corr(int nb, const double* __restrict__ cpart, const float* __restrict__ w,
                           float* __restrict__ cvec, double* __restrict__ rz_slot) {
  __shared__ double sp[4][kDefK];
  __shared__ double sh[kDefK];
  const int j = threadIdx.x & (kDefK - 1), part = threadIdx.x >> 6;
  double s4 = 0.0;
  for (int b = part; b < nb; b += 4) s4 += cpart[(int64_t)b * kDefK + j];
  sp[part][j] = s4;
  __syncthreads();
  if (threadIdx.x < kDefK) {
    const double s = ((sp[0][j] + sp[1][j]) + sp[2][j]) + sp[3][j];
    cvec[j] = (float)s;
    sh[j] = (double)w[j] * s * s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kDefK; ++q) t += sh[q];
    rz_slot[0] += t;
  }
}

// z = M^-1 r + Yw c; p = z + beta p; pd = d o p.  beta = rz_new / rz_prev from
// the CG's per-block partial slots (each block sums them in the same order),
// or 0 when part is null.
__global__ void k_df1_update(int64_t n, const float* __restrict__ minv, const float* __restrict__ dv,
                             const float* __restrict__ Yw, const float* __restrict__ cvec,
                             const double* __restrict__ part, int G, int prev, int next,
                             const float* __restrict__ r, float* __restrict__ p,
                             float* __restrict__ pd) {
  __shared__ float cs[kDefK];
  __shared__ float sh_beta;
  if (threadIdx.x < kDefK) cs[threadIdx.x] = cvec[threadIdx.x];
  if (threadIdx.x < 32) {  // warp 0: the same fixed-order sums in every block
    double rzp = 0.0, rzn = 0.0;
    if (part)
      for (int k = threadIdx.x; k < G; k += 32) {
        rzp += part[prev * G + k];
        rzn += part[next * G + k];
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      rzp += __shfl_xor_sync(0xffffffffu, rzp, off);
      rzn += __shfl_xor_sync(0xffffffffu, rzn, off);
    }
    if (threadIdx.x == 0) sh_beta = (part && rzp > 0) ? (float)(rzn / rzp) : 0.f;
  }
  __syncthreads();
  const float beta = sh_beta;
  // eight lanes per row, eight of the row's 64 products each, summed by shuffles
  // (a warp takes four rows per pass, so its shuffles never diverge)
  const int l8 = threadIdx.x & 7, sub = (threadIdx.x & 31) >> 3;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = 4 * gw; base < n; base += 4 * nwarp) {
    const int64_t i = base + sub;
    const bool v = i < n;
    float z = 0.f;
    if (v) {
      const float4* y4 = reinterpret_cast<const float4*>(Yw + i * kDefK + 8 * l8);
      const float4 a = __ldg(y4), b = __ldg(y4 + 1);
      const float* c8 = cs + 8 * l8;
      z = fmaf(a.x, c8[0], fmaf(a.y, c8[1], fmaf(a.z, c8[2], fmaf(a.w, c8[3],
          fmaf(b.x, c8[4], fmaf(b.y, c8[5], fmaf(b.z, c8[6], b.w * c8[7])))))));
    }
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    if (v && l8 == 0) {
      const float pi = minv[i] * r[i] + z + beta * p[i];
      p[i] = pi;
      pd[i] = dv[i] * pi;
    }
  }
}

// ---------------------------------------------------------------- host LA
// Cholesky G = L L^T (in place, lower), FP64; false if not positive definite.
static bool chol(std::vector<double>& G, int k) {
  for (int j = 0; j < k; ++j) {
    double d = G[j * k + j];
    for (int p = 0; p < j; ++p) d -= G[j * k + p] * G[j * k + p];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    G[j * k + j] = d;
    for (int i = j + 1; i < k; ++i) {
      double s = G[i * k + j];
      for (int p = 0; p < j; ++p) s -= G[i * k + p] * G[j * k + p];
      G[i * k + j] = s / d;
    }
    for (int i = 0; i < j; ++i) G[i * k + j] = 0.0;
  }
  return true;
}

// Inverse of L^T (upper triangular) as a row-major k x k matrix U with
// W_new = W U orthonormal when W^T W = L L^T.
static std::vector<double> inv_lt(const std::vector<double>& L, int k) {
  // solve L^T U = I column by column (back substitution)
  std::vector<double> U(k * k, 0.0);
  for (int col = 0; col < k; ++col) {
    for (int i = k - 1; i >= 0; --i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int p = i + 1; p < k; ++p) s -= L[p * k + i] * U[p * k + col];
      U[i * k + col] = s / L[i * k + i];
    }
  }
  return U;
}

// Cyclic Jacobi eigen-solver for a symmetric k x k matrix (row-major, FP64):
// A = S diag(lambda) S^T; S columns are the eigenvectors.
static void jacobi_eig(std::vector<double> A, int k, std::vector<double>& lambda,
                       std::vector<double>& S) {
  S.assign(k * k, 0.0);
  for (int i = 0; i < k; ++i) S[i * k + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        tot += A[i * k + j] * A[i * k + j];
        if (i != j) off += A[i * k + j] * A[i * k + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[p * k + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[p * k + p], aqq = A[q * k + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < k; ++r) {  // A <- A J (columns p, q)
          const double arp = A[r * k + p], arq = A[r * k + q];
          A[r * k + p] = cs * arp - sn * arq;
          A[r * k + q] = sn * arp + cs * arq;
        }
        for (int r = 0; r < k; ++r) {  // A <- J^T A (rows p, q)
          const double apr = A[p * k + r], aqr = A[q * k + r];
          A[p * k + r] = cs * apr - sn * aqr;
          A[q * k + r] = sn * apr + cs * aqr;
        }
        for (int r = 0; r < k; ++r) {  // S <- S J
          const double srp = S[r * k + p], srq = S[r * k + q];
          S[r * k + p] = cs * srp - sn * srq;
          S[r * k + q] = sn * srp + cs * srq;
        }
      }
  }
  lambda.resize(k);
  for (int i = 0; i < k; ++i) lambda[i] = A[i * k + i];
}

// ---------------------------------------------------------------- host
static int eg(gm_ctx* c, int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), 16 * sm_count(c)));
}

// G = X^T Z (FP64) brought to the host
static gm_status gram(gm_ctx* c, Deflation& F, const float* X, const float* Z,
                      std::vector<double>& h) {
  const int nb = (int)ceil_div(F.n, 64);
  if (!ensure(c, F.Gp, (size_t)nb * kDefK * kDefK * sizeof(double)))
    return set_error(c, GM_E_NOMEM, "deflation Gram partials");
  GM_PROF(c, "k_df_gram");
  k_df_gram<<<nb, 256, 0, c->stream>>>(F.n, X, Z, (double*)F.Gp.p);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_df_gram_sum");
  k_df_gram_sum<<<kDefK * kDefK / 256, 256, 0, c->stream>>>(nb, (const double*)F.Gp.p,
                                                            (double*)F.G.p);
  GM_LAUNCH_CHECK(c);
  h.resize(kDefK * kDefK);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), F.G.p, h.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

// Out = In M (M: k x k FP64 on the host, applied in FP32)
static gm_status right_mul(gm_ctx* c, Deflation& F, const float* In,
                           const std::vector<double>& M, float* Out) {
  std::vector<float> m(M.begin(), M.end());
  GM_CUDA_CHECK(c, cudaMemcpyAsync(F.Mk.p, m.data(), m.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, c->stream));
  GM_PROF(c, "k_df_right");
  k_df_right<<<eg(c, F.n * kDefK), 256, 0, c->stream>>>(F.n, In, (const float*)F.Mk.p, Out);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));  // m lives on this stack frame
  return GM_OK;
}

// In <- orthonormal basis of span(In) (two Cholesky-QR passes); Tmp scratch
static gm_status orth(gm_ctx* c, Deflation& F, float* In, float* Tmp, bool* ok) {
  std::vector<double> G;
  float* src = In;
  float* dst = Tmp;
  for (int pass = 0; pass < 2; ++pass) {
    gm_status s = gram(c, F, src, src, G);
    if (s != GM_OK) return s;
    if (!chol(G, kDefK)) {
      *ok = false;
      return GM_OK;
    }
    s = right_mul(c, F, src, inv_lt(G, kDefK), dst);
    if (s != GM_OK) return s;
    std::swap(src, dst);
  }
  *ok = true;  // two passes: the result is back in In
  return GM_OK;
}

gm_status deflate_prepare(gm_ctx* c, const float* dv, const float* minv) {
  Deflation& F = D(c);
  const int64_t n = c->n;
  const size_t nk = (size_t)n * kDefK * sizeof(float);
  if (F.n != n) {
    F.n = n;
    F.have_v = false;
  }
  // partial rows of a k-column panel product: one per tile block or per
  // block row of the CUDA-core kernels (at most ceil(n / 8))
  const int64_t npart = std::max<int64_t>(c->tc_nblk, ceil_div(n, 8)) + 1;
  F.ready = false;
  if (!ensure(c, F.V, nk) || !ensure(c, F.W, nk) || !ensure(c, F.Y, nk) || !ensure(c, F.Yw, nk) ||
      !ensure(c, F.P, nk) || !ensure(c, F.PD, nk) || !ensure(c, F.Q, nk) ||
      !ensure(c, F.part, (size_t)npart * kDefK * sizeof(double)) ||
      !ensure(c, F.G, kDefK * kDefK * sizeof(double)) ||
      !ensure(c, F.Mk, kDefK * kDefK * sizeof(float)) || !ensure(c, F.ms, n * sizeof(float)) ||
      !ensure(c, F.wv, kDefK * sizeof(float)))
    return set_error(c, GM_E_NOMEM, "deflation vectors");
  float *V = (float*)F.V.p, *Wb = (float*)F.W.p, *P = (float*)F.P.p, *PD = (float*)F.PD.p,
        *Q = (float*)F.Q.p, *ms = (float*)F.ms.p;
  cudaStream_t st = c->stream;
  GM_PROF(c, "k_df_ms");
  k_df_ms<<<eg(c, n), 256, 0, st>>>(n, minv, ms);
  GM_LAUNCH_CHECK(c);
  if (!F.have_v) {
    GM_PROF(c, "k_df_init");
    k_df_init<<<eg(c, n * kDefK), 256, 0, st>>>(n, V);
    GM_LAUNCH_CHECK(c);
    bool ok = false;
    gm_status s = orth(c, F, V, Wb, &ok);
    if (s != GM_OK) return s;
    if (!ok) return GM_OK;  // no deflation this refresh (plain Jacobi)
  }
  // W = B~ V = ms o (B (ms o V))
  auto apply = [&](const float* X, float* Out) -> gm_status {
    GM_PROF(c, "k_df_scale_in");
    k_df_scale_in<<<eg(c, n * kDefK), 256, 0, st>>>(n, ms, dv, X, P, PD);
    GM_LAUNCH_CHECK(c);
    gm_status s = panel_apply_B_f32(c, kDefK, dv, P, PD, Q, (double*)F.part.p);
    if (s != GM_OK) return s;
    GM_PROF(c, "k_df_scale_out");
    k_df_scale_out<<<eg(c, n * kDefK), 256, 0, st>>>(n, ms, Q, Out);
    GM_LAUNCH_CHECK(c);
    return GM_OK;
  };
  // (six warm-started steps instead of three gave the same CG iteration
  // counts on the 20,000-star bench)
  const int iters = F.have_v ? kDefItersWarm : kDefIters;
  for (int it = 0; it < iters; ++it) {
    gm_status s = apply(V, Wb);
    if (s != GM_OK) return s;
    bool ok = false;
    s = orth(c, F, Wb, V, &ok);  // Wb <- orth(Wb), V used as scratch
    if (s != GM_OK) return s;
    if (!ok) {  // V may be clobbered: restart from a fresh block next refresh
      F.have_v = false;
      return GM_OK;
    }
    std::swap(F.V, F.W);
    V = (float*)F.V.p;
    Wb = (float*)F.W.p;
  }
  // Rayleigh-Ritz on span V: H = V^T B~ V, H = S diag(theta) S^T, V <- V S
  gm_status s = apply(V, Wb);
  if (s != GM_OK) return s;
  std::vector<double> H, S;
  s = gram(c, F, V, Wb, H);
  if (s != GM_OK) return s;
  for (int a = 0; a < kDefK; ++a)
    for (int b = a + 1; b < kDefK; ++b) {
      const double m = 0.5 * (H[a * kDefK + b] + H[b * kDefK + a]);
      H[a * kDefK + b] = H[b * kDefK + a] = m;
    }
  jacobi_eig(H, kDefK, F.theta, S);
  s = right_mul(c, F, V, S, Wb);
  if (s != GM_OK) return s;
  std::swap(F.V, F.W);
  V = (float*)F.V.p;
  F.have_v = true;
  std::vector<float> w(kDefK);
  for (int j = 0; j < kDefK; ++j) {
    const double th = F.theta[j];
    w[j] = th > 0 ? (float)(1.0 / th - 1.0) : 0.f;  // theta <= 0 cannot occur for SPD B
  }
  GM_CUDA_CHECK(c, cudaMemcpyAsync(F.wv.p, w.data(), kDefK * sizeof(float), cudaMemcpyHostToDevice,
                                   st));
  GM_PROF(c, "k_df_make_y");
  k_df_make_y<<<eg(c, n * kDefK), 256, 0, st>>>(n, ms, V, (const float*)F.wv.p, (float*)F.Y.p,
                                                (float*)F.Yw.p);
  GM_LAUNCH_CHECK(c);
  // tensor-core form of the panel step: BF16 pieces of Y^T and Yw
  F.tc = false;
  const char* e = std::getenv("GM_DEFLATE_TC");
  if (c->tc_nblk > 0 && !(e && e[0] == '0')) {
    if (!ensure(c, F.yimg, dtc_yimg_bytes(n)) || !ensure(c, F.ywimg, dtc_rowimg_bytes(n)))
      return set_error(c, GM_E_NOMEM, "deflation images");
    gm_status si = dtc_images(c, n, (const float*)F.Y.p, (const float*)F.Yw.p, F.yimg.p,
                              F.ywimg.p);
    if (si != GM_OK) return si;
    F.tc = true;
  }
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));  // w lives on this stack frame
  F.ready = true;
  return GM_OK;
}

bool deflate_ready(gm_ctx* c) { return c->defl && c->defl->ready; }

gm_status deflate_rhs(gm_ctx* c, int R, const float* Rr, double* corr_row) {
  Deflation& F = D(c);
  const int64_t n = c->n;
  const int nrb = (int)ceil_div(n, kDefRows);
  if (!ensure(c, F.Cp, (size_t)nrb * kDefK * R * sizeof(float)) ||
      !ensure(c, F.C, (size_t)kDefK * R * sizeof(float)))
    return set_error(c, GM_E_NOMEM, "deflation projections");
  GM_PROF(c, "k_df_yt_r");
  k_df_yt_r<<<dim3((unsigned)ceil_div(R, 128), (unsigned)nrb), 256, 0, c->stream>>>(
      n, R, (const float*)F.Y.p, Rr, (float*)F.Cp.p);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_df_sum");
  k_df_sum<<<eg(c, (int64_t)kDefK * R), 256, 0, c->stream>>>(R, nrb, (const float*)F.Cp.p,
                                                             (float*)F.C.p);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_df_corr");
  k_df_corr<<<(int)ceil_div(R, 128), 128, 0, c->stream>>>(R, (const float*)F.C.p,
                                                          (const float*)F.wv.p, corr_row);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status deflate_update(gm_ctx* c, int R, int nbx, const float* minv, const float* dv,
                         const double* beta, const int* active, const float* Rr, float* P,
                         float* PD) {
  Deflation& F = D(c);
  (void)nbx;
  const int smem = (kDefK * 64 + kDefK * 128) * (int)sizeof(float);  // 48 KB
  GM_PROF(c, "k_df_update");
  k_df_update<<<dim3((unsigned)ceil_div(R, 128), (unsigned)ceil_div(c->n, 64)), 256, smem,
                c->stream>>>(c->n, R, minv, dv, beta, active, Rr, (const float*)F.Yw.p,
                             (const float*)F.C.p, P, PD);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

bool deflate_tc(gm_ctx* c) { return c->defl && c->defl->ready && c->defl->tc; }

int deflate_tc_chunks(gm_ctx* c, int R) { return dtc_chunks(c, c->n, R); }

gm_status deflate_step_tc(gm_ctx* c, int R, int nch, const double* alpha, const float* minv,
                          float* X, float* Rr, const float* P, const float* Q, double* part_rz,
                          double* part_rr, double* corr8) {
  Deflation& F = D(c);
  if (!ensure(c, F.Cp2, (size_t)2 * nch * kDefK * R * sizeof(float)) ||
      !ensure(c, F.cimg, dtc_cimg_bytes(R)))
    return set_error(c, GM_E_NOMEM, "deflation projections");
  return dtc_step(c, c->n, R, nch, F.yimg.p, alpha, minv, X, Rr, P, Q, part_rz, part_rr,
                  (float*)F.Cp2.p, (const float*)F.wv.p, F.cimg.p, corr8);
}

gm_status deflate_update_tc(gm_ctx* c, int R, const float* minv, const float* dv,
                            const double* beta, const int* active, const float* Rr, float* P,
                            float* PD, bool planes) {
  Deflation& F = D(c);
  uint16_t* pl = nullptr;
  if (planes) {
    if (!ensure(c, c->tc_planes, (size_t)c->n * R * 3 * sizeof(uint16_t)))
      return set_error(c, GM_E_NOMEM, "BF16 planes of the panel");
    pl = (uint16_t*)c->tc_planes.p;
  }
  return dtc_update(c, c->n, R, F.ywimg.p, F.cimg.p, minv, dv, beta, active, Rr, P, PD, pl);
}

// Single right-hand side: c = Y^T r, add sum_j w_j c_j^2 to rz_slot[0]
gm_status deflate1_rhs(gm_ctx* c, const float* r, double* rz_slot) {
  Deflation& F = D(c);
  const int nb = 2 * sm_count(c);
  if (!ensure(c, F.cpart1, (size_t)nb * kDefK * sizeof(double)) ||
      !ensure(c, F.c1, kDefK * sizeof(float)))
    return set_error(c, GM_E_NOMEM, "deflation projections");
  GM_PROF(c, "k_df1_part");
  k_df1_part<<<nb, 256, 0, c->stream>>>(c->n, (const float*)F.Y.p, r, (double*)F.cpart1.p);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_df1_corr");
  k_df1_corr<<<1, 4 * kDefK, 0, c->stream>>>(nb, (const double*)F.cpart1.p, (const float*)F.wv.p,
                                         (float*)F.c1.p, rz_slot);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

// p = M^-1 r + Yw c + beta p, pd = d o p (c from deflate1_rhs; beta from the
// partial slots prev / next of part, or 0 when part is null)
gm_status deflate1_update(gm_ctx* c, const float* minv, const float* dv, const double* part,
                          int G, int prev, int next, const float* r, float* p, float* pd) {
  Deflation& F = D(c);
  GM_PROF(c, "k_df1_update");
  k_df1_update<<<eg(c, 8 * c->n), 256, 0, c->stream>>>(c->n, minv, dv, (const float*)F.Yw.p,
                                                    (const float*)F.c1.p, part, G, prev, next,
                                                    r, p, pd);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm
