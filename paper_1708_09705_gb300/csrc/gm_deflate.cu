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
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kDefK = 64;          // deflation vectors
constexpr int kDefIters = 8;       // subspace-iteration steps per refresh
constexpr int kDefRows = 256;      // rows per block of the Y^T R kernel

struct Deflation {
  int64_t n = 0;
  bool have_v = false;
  Buffer V, W, Y, Yw;              // n x k FP32 (row-major)
  Buffer P, PD, Q;                 // n x k panel product buffers
  Buffer part;                     // panel-product partials
  Buffer G;                        // k x k FP64 Gram / projection
  Buffer Mk;                       // k x k FP32 matrix applied on the right
  Buffer ms;                       // n: M^-1/2
  Buffer Cp, C;                    // Y^T R: partials per row block, and the sum (k x R)
  Buffer wv;                       // k weights 1/theta - 1 (FP32)
  std::vector<double> theta;       // Ritz values of this refresh
  bool ready = false;              // Y, Yw, wv valid for this refresh
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

// G[a][b] = sum_i X[i][a] Z[i][b] in FP64: block per a, thread per b with a
// fixed row order (the block's 64 threads walk the rows together).
__global__ void k_df_gram(int64_t n, const float* __restrict__ X, const float* __restrict__ Z,
                          double* __restrict__ G) {
  const int a = blockIdx.x, b = threadIdx.x;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += (double)X[i * kDefK + a] * (double)Z[i * kDefK + b];
  G[a * kDefK + b] = s;
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

// Cp[rb][j][c] = sum over the block's rows i of Y[i][j] R[i][c]; thread per
// column c, the block's rows staged 32 at a time in shared memory.
__global__ void __launch_bounds__(128) k_df_yt_r(int64_t n, int R, const float* __restrict__ Y,
                                                 const float* __restrict__ Rr,
                                                 float* __restrict__ Cp) {
  __shared__ __align__(16) float ys[32][kDefK];
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int64_t rb = blockIdx.y;
  const int64_t i0 = rb * kDefRows, i1 = min(i0 + kDefRows, n);
  float acc[kDefK];
#pragma unroll
  for (int j = 0; j < kDefK; ++j) acc[j] = 0.f;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    const int cnt = (int)min((int64_t)32, i1 - ib);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * kDefK; e += blockDim.x) {
      const int r = e / kDefK, j = e - r * kDefK;
      ys[r][j] = r < cnt ? Y[(ib + r) * kDefK + j] : 0.f;
    }
    __syncthreads();
    if (c < R) {
      for (int r = 0; r < cnt; ++r) {
        const float v = Rr[(ib + r) * R + c];
        const float4* y4 = reinterpret_cast<const float4*>(ys[r]);
#pragma unroll
        for (int q = 0; q < kDefK / 4; ++q) {
          const float4 y = y4[q];
          acc[4 * q] = fmaf(y.x, v, acc[4 * q]);
          acc[4 * q + 1] = fmaf(y.y, v, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(y.z, v, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(y.w, v, acc[4 * q + 3]);
        }
      }
    }
  }
  if (c < R) {
#pragma unroll
    for (int j = 0; j < kDefK; ++j) Cp[(rb * kDefK + j) * R + c] = acc[j];
  }
}

// C[j][c] = sum_rb Cp[rb][j][c] (fixed order); corr[c] = sum_j w_j C[j][c]^2
__global__ void k_df_sum(int R, int nrb, const float* __restrict__ Cp, const float* __restrict__ w,
                         float* __restrict__ C, double* __restrict__ corr) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    double cs = 0.0;
    for (int j = 0; j < kDefK; ++j) {
      float s = 0.f;
      for (int rb = 0; rb < nrb; ++rb) s += Cp[((int64_t)rb * kDefK + j) * R + c];
      C[(int64_t)j * R + c] = s;
      cs += (double)w[j] * (double)s * (double)s;
    }
    corr[c] = cs;
  }
}

// P = M^-1 R + Yw C + beta P (columns active, or all when active is null),
// PD = d o P.  Thread per column (its 64 C values in registers), rows strided.
__global__ void __launch_bounds__(256) k_df_update(int64_t n, int R, const float* __restrict__ minv,
                                                   const float* __restrict__ dv,
                                                   const double* __restrict__ beta,
                                                   const int* __restrict__ active,
                                                   const float* __restrict__ Rr,
                                                   const float* __restrict__ Yw,
                                                   const float* __restrict__ C,
                                                   float* __restrict__ P, float* __restrict__ PD) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  if (c >= R) return;
  if (active && !active[c]) return;  // frozen column: P is never read with alpha != 0
  const float be = beta ? (float)beta[c] : 0.f;
  float cc[kDefK];
#pragma unroll
  for (int j = 0; j < kDefK; ++j) cc[j] = C[(int64_t)j * R + c];
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = w; i < n; i += nw) {
    const float4* y4 = reinterpret_cast<const float4*>(Yw + i * kDefK);
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < kDefK / 4; ++q) {
      const float4 y = __ldg(y4 + q);
      z = fmaf(y.x, cc[4 * q], z);
      z = fmaf(y.y, cc[4 * q + 1], z);
      z = fmaf(y.z, cc[4 * q + 2], z);
      z = fmaf(y.w, cc[4 * q + 3], z);
    }
    const int64_t k = i * R + c;
    const float p = minv[i] * Rr[k] + z + be * P[k];
    P[k] = p;
    PD[k] = dv[i] * p;
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
  GM_PROF(c, "k_df_gram");
  k_df_gram<<<kDefK, kDefK, 0, c->stream>>>(F.n, X, Z, (double*)F.G.p);
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
  for (int it = 0; it < kDefIters; ++it) {
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
  k_df_yt_r<<<dim3((unsigned)ceil_div(R, 128), (unsigned)nrb), 128, 0, c->stream>>>(
      n, R, (const float*)F.Y.p, Rr, (float*)F.Cp.p);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_df_sum");
  k_df_sum<<<(int)ceil_div(R, 128), 128, 0, c->stream>>>(R, nrb, (const float*)F.Cp.p,
                                                         (const float*)F.wv.p, (float*)F.C.p,
                                                         corr_row);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status deflate_update(gm_ctx* c, int R, int nbx, const float* minv, const float* dv,
                         const double* beta, const int* active, const float* Rr, float* P,
                         float* PD) {
  Deflation& F = D(c);
  GM_PROF(c, "k_df_update");
  k_df_update<<<dim3((unsigned)nbx, (unsigned)(R / 32)), 256, 0, c->stream>>>(
      c->n, R, minv, dv, beta, active, Rr, (const float*)F.Yw.p, (const float*)F.C.p, P, PD);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm
