// Tensor-core kernels of the deflated preconditioner of the FP32 variance
// panels.
//
// Each CG iteration on a panel of R right-hand sides applies the spectral
// preconditioner M_d^-1 = M^-1 + Y (Theta^-1 - I) Y^T (Saad, Iterative Methods
// for Sparse Linear Systems, Sect. 9.6) to the updated residuals R':
// C = Y^T R' (64 x R) and P = M^-1 R' + Yw C + beta P, Yw = Y (Theta^-1 - I).
// Both are dense contractions (inner dimension n and 64); here they run on
// the tcgen05 tensor cores with every FP32 operand split into three BF16
// pieces (x = x1 + x2 + x3 exactly; the six piece products down to 2^-16 of
// the leading one give FP32-grade products, as in the tile product).
//
// k_dtc_step fuses the CG update of the panel with C's partial sums.  CTA =
// (128 panel columns, a chunk of 16-row K-steps).  Per K-step the four
// producer warps load X, P, R and Q of their rows, write X + alpha P and
// R' = R - alpha Q, accumulate r'^T M^-1 r' and r'^T r' per column, and store
// the three BF16 pieces of R' into a 128-byte-swizzled MN-major B tile; thread
// 0 bulk-copies the K-step's image of the pieces of Y^T; one thread of the
// fifth warp issues four MMAs (M = 128, N = 128, K = 16) with the pieces of Y^T
// stacked in M: [Y1; Y2] R'3, [Y1; Y2] R'2, [Y1; Y2] R'1 and [Y3; 0] R'1.  The
// accumulator's two 64-row halves then hold Y1 R' + Y3 R'1 and Y2 R' (seven
// of the nine piece products, the six of the split among them) and are
// written as two partial rows of C per chunk.
// k_dtc_sum adds the partial rows in a fixed order, forms the deflation term
// sum_j w_j C_jc^2 of r^T z (eight partial rows, FP64) and writes the K-major
// images of C's pieces.
// k_dtc_update: CTA = (128 rows, 128 columns); bulk copies of the 128 x 64
// images of Yw's pieces and the 128 x 64 images of C^T's pieces, 24 MMAs (six
// products x four K-steps of 16), epilogue P = M^-1 R' + acc + beta P on
// active columns (frozen columns keep P) and D P, either in FP32 or directly
// as the three BF16 planes the tile product copies its B operand from.  The
// accumulator rows go through shared memory first, so that every global
// access of the epilogue covers whole row segments (16 lanes x 16 bytes).
#include <algorithm>
#include <cstdlib>

#include "gm_internal.cuh"
#include "gm_tcgen05.cuh"

namespace gm {

constexpr int kDk = 64;  // deflation vectors

// ---- step kernel
constexpr int kS1Cols = 128;                       // panel columns per CTA (N)
constexpr int kS1Ring = 3;
constexpr int kS1Prod = 128;                       // producer threads
constexpr int kS1Threads = kS1Prod + 32;
constexpr int kS1B = 16 * kS1Cols * 2;             // one piece of the 16 x 128 R' tile (4 KB)
constexpr int kS1A = kDk * 16 * 2;                 // one piece of the 64 x 16 Y^T tile (2 KB)
constexpr int kS1Img = 3 * kS1A;                   // Y^T image of one K-step (6 KB)
constexpr int kS1Stage = 3 * kS1B + 4 * kS1A;      // + a zero block under Y3 (20 KB)
constexpr int kS1Smem = kS1Ring * kS1Stage + 1024;  // + alignment of the swizzled tiles

// ---- update kernel
constexpr int kU2Piece = 128 * kDk * 2;            // one piece of a 128 x 64 image (16 KB)
constexpr int kU2Img = 3 * kU2Piece;
constexpr int kU2Smem = 2 * kU2Img + 128;
constexpr int kU2Stg = 68;  // floats per staged accumulator row (64 + 4: no bank conflicts)

// byte offset of R' element (k, n) in one piece of the 16 x 128 B tile: the
// MN-major 128-byte-swizzle layout, atoms of 8 k-rows x 64 columns (1 KB),
// atoms along n 1 KB apart, k-groups 2 KB apart
__host__ __device__ __forceinline__ int s1_boff(int k, int n) {
  return (n >> 6) * 1024 + (k >> 3) * 2048 + (k & 7) * 128 + ((((n >> 3) & 7) ^ (k & 7)) << 4) +
         (n & 7) * 2;
}

// byte offset of element (row, k) in a K-major no-swizzle image with 16
// columns of k (8 x 16-byte core matrices, k-adjacent 128 B apart, 8-row
// groups 256 B apart)
__host__ __device__ __forceinline__ int k16_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// the same with 64 columns of k (8-row groups 1 KB apart)
__host__ __device__ __forceinline__ int k64_off(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------- images
// Y^T pieces per K-step of 16 rows: piece p of K-step ks at
// img + ks * kS1Img + p * kS1A, element (j, k) = piece of Y[16 ks + k][j]
// (zero past row n).  Thread per (K-step, j, half of the K-step).
__global__ void k_dtc_img_y(int64_t n, int64_t nks, const float* __restrict__ Y,
                            unsigned char* __restrict__ img) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nks * kDk * 2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ks = e / (kDk * 2);
    const int rem = (int)(e - ks * kDk * 2), j = rem >> 1, k8 = rem & 1;
    float v[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int64_t i = 16 * ks + 8 * k8 + kk;
      v[kk] = i < n ? Y[i * kDk + j] : 0.f;
    }
    uint4 p1, p2, p3;
    tg::split3x8(v, p1, p2, p3);
    unsigned char* dst = img + ks * kS1Img + k16_off(j, 8 * k8);
    *reinterpret_cast<uint4*>(dst) = p1;
    *reinterpret_cast<uint4*>(dst + kS1A) = p2;
    *reinterpret_cast<uint4*>(dst + 2 * kS1A) = p3;
  }
}

// Pieces of the rows of an n x 64 matrix per block of 128 rows: piece p of
// block b at img + b * kU2Img + p * kU2Piece, K-major 128 x 64 (zero past row
// n).  Thread per (block, row, 8 columns).
__global__ void k_dtc_img_rows(int64_t n, int64_t nblk, const float* __restrict__ A,
                               unsigned char* __restrict__ img) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nblk * 128 * 8;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e >> 10;
    const int r = (int)((e >> 3) & 127), k8 = (int)(e & 7);
    const int64_t i = b * 128 + r;
    float v[8];
    if (i < n) {
      const float4 a = *reinterpret_cast<const float4*>(A + i * kDk + 8 * k8);
      const float4 c = *reinterpret_cast<const float4*>(A + i * kDk + 8 * k8 + 4);
      v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = c.x, v[5] = c.y, v[6] = c.z,
      v[7] = c.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = 0.f;
    }
    uint4 p1, p2, p3;
    tg::split3x8(v, p1, p2, p3);
    unsigned char* dst = img + b * kU2Img + k64_off(r, 8 * k8);
    *reinterpret_cast<uint4*>(dst) = p1;
    *reinterpret_cast<uint4*>(dst + kU2Piece) = p2;
    *reinterpret_cast<uint4*>(dst + 2 * kU2Piece) = p3;
  }
}

// ---------------------------------------------------------------- step
// One producer thread's loads of a K-step.
struct StepRegs {
  float4 r[4], x[4], p[4], q[4];
  float m[4];
  int v;  // bit h: row h of the K-step is a row of the panel
};

// alpha null: C's partial rows of R only (X, R untouched, no rz / rr).
// Three CTAs per SM (registers and shared memory); a second K-step of loads
// in flight per producer needed ~230 registers (one CTA per SM) or spilled
// at two CTAs per SM, and was slower either way.
__global__ void __launch_bounds__(kS1Threads, 3) k_dtc_step(
    int64_t n, int R, int kpc, const unsigned char* __restrict__ yimg,
    const double* __restrict__ alpha, const float* __restrict__ minv, float* __restrict__ X,
    float* __restrict__ Rr, const float* __restrict__ P, const float* __restrict__ Q,
    double* __restrict__ part_rz, double* __restrict__ part_rr, float* __restrict__ Cp,
    unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t fullA[kS1Ring], fullB[kS1Ring], empty[kS1Ring];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ double sh_rz[4][kS1Cols], sh_rr[4][kS1Cols];
  volatile int* abort_v = &abort_flag;
  // the swizzle pattern follows the address bits: stages start on 1 KB
  unsigned char* sm = smem_raw + ((1024u - (tg::smem(smem_raw) & 1023u)) & 1023u);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int c0 = blockIdx.x * kS1Cols;
  const int chunk = blockIdx.y;
  const int64_t nks_tot = (n + 15) / 16;
  const int64_t ks0 = (int64_t)chunk * kpc;
  const int64_t nks = nks_tot - ks0 < 0 ? 0 : (nks_tot - ks0 < kpc ? nks_tot - ks0 : kpc);
  const bool upd = alpha != nullptr;

  if (t == 0) {
    abort_flag = 0;
    for (int q = 0; q < kS1Ring; ++q) {
      tg::mbar_init(tg::smem(&fullA[q]), 1);
      tg::mbar_init(tg::smem(&fullB[q]), kS1Prod);
      tg::mbar_init(tg::smem(&empty[q]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the zero rows under Y3 in every stage (never overwritten)
  for (int e = t; e < kS1Ring * (kS1A / 16); e += kS1Threads) {
    const int s = e / (kS1A / 16), q = e - s * (kS1A / 16);
    *reinterpret_cast<uint4*>(sm + s * kS1Stage + 3 * kS1B + 3 * kS1A + 16 * q) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        tg::smem(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // columns 4 lane .. 4 lane + 3 of the CTA's 128, rows warp + 4 h (h < 4) of
  // each K-step: every load of a warp is one 512-byte row segment
  const int col = c0 + 4 * lane;
  const bool vcol = col < R;  // R is a multiple of 32: 4 columns all in or all out
  PartialSum<float> rz[4], rr[4];

  if (warp < 4) {
    float a[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = (upd && vcol) ? (float)alpha[col + e] : 0.f;
    int64_t issued = 0;
    // the loads of one K-step: the thread's four row segments of R (and X,
    // P, Q when updating)
    auto load = [&](int64_t ks, StepRegs& S) {
      S.v = 0;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int64_t i = 16 * (ks0 + ks) + warp + 4 * h;
        const bool vh = vcol && i < n;
        S.v |= vh ? 1 << h : 0;
        S.m[h] = 0.f;
        S.r[h] = S.x[h] = S.p[h] = S.q[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (vh) {
          const int64_t at = i * R + col;
          S.r[h] = *reinterpret_cast<const float4*>(Rr + at);
          if (upd) {
            S.x[h] = *reinterpret_cast<const float4*>(X + at);
            S.p[h] = __ldcs(reinterpret_cast<const float4*>(P + at));
            S.q[h] = __ldcs(reinterpret_cast<const float4*>(Q + at));
            S.m[h] = minv[i];
          }
        }
      }
    };
    // update, partial sums, BF16 pieces of R' into stage ks % ring; false
    // when a wait gave up
    auto produce = [&](int64_t ks, const StepRegs& S) -> bool {
      const int s = (int)(ks % kS1Ring);
      const int64_t use = ks / kS1Ring;
      if (use > 0 && !tg::wait(tg::smem(&empty[s]), (uint32_t)((use - 1) & 1), abort_v)) {
        abort_flag = 1;
        return false;
      }
      unsigned char* sB = sm + s * kS1Stage;
      if (t == 0) {
        tg::arrive_expect_tx(tg::smem(&fullA[s]), kS1Img);
        tg::bulk_g2s(tg::smem(sB + 3 * kS1B), yimg + (ks0 + ks) * kS1Img, kS1Img,
                     tg::smem(&fullA[s]));
        ++issued;
      }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int kr = warp + 4 * h;
        float rv[4] = {S.r[h].x, S.r[h].y, S.r[h].z, S.r[h].w};
        if (upd && (S.v >> h & 1)) {
          const int64_t at = (16 * (ks0 + ks) + kr) * R + col;
          const float xv[4] = {S.x[h].x, S.x[h].y, S.x[h].z, S.x[h].w};
          const float pv[4] = {S.p[h].x, S.p[h].y, S.p[h].z, S.p[h].w};
          const float qv[4] = {S.q[h].x, S.q[h].y, S.q[h].z, S.q[h].w};
          float xn[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xn[e] = xv[e] + a[e] * pv[e];
            rv[e] = rv[e] - a[e] * qv[e];
            rz[e].add(rv[e] * (S.m[h] * rv[e]));
            rr[e].add(rv[e] * rv[e]);
          }
          *reinterpret_cast<float4*>(X + at) = make_float4(xn[0], xn[1], xn[2], xn[3]);
          *reinterpret_cast<float4*>(Rr + at) = make_float4(rv[0], rv[1], rv[2], rv[3]);
        }
        uint2 p1, p2, p3;
        tg::split3x4(rv, p1, p2, p3);
        const int off = s1_boff(kr, 4 * lane);
        *reinterpret_cast<uint2*>(sB + off) = p1;
        *reinterpret_cast<uint2*>(sB + kS1B + off) = p2;
        *reinterpret_cast<uint2*>(sB + 2 * kS1B + off) = p3;
      }
      // the pieces were written through the generic proxy; the MMAs read
      // them through the async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tg::arrive(tg::smem(&fullB[s]));
      return true;
    };
    StepRegs A;
    for (int64_t ks = 0; ks < nks; ++ks) {
      load(ks, A);
      if (!produce(ks, A)) break;
    }
    if (t == 0 && *abort_v) {  // bounded waits for the bulk copies still in flight
      for (int qq = 0; qq < kS1Ring; ++qq) {
        const int64_t na = issued > qq ? (issued - 1 - qq) / kS1Ring + 1 : 0;
        if (na > 0) tg::wait(tg::smem(&fullA[qq]), (uint32_t)((na - 1) & 1), nullptr);
      }
    }
  } else if (warp == 4 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idesc = tg::idesc_bf16(128, kS1Cols, false, true);
    int64_t done = 0;
    for (int64_t ks = 0; ks < nks; ++ks) {
      const int s = (int)(ks % kS1Ring);
      const uint32_t par = (uint32_t)((ks / kS1Ring) & 1);
      if (!tg::wait(tg::smem(&fullA[s]), par, abort_v) ||
          !tg::wait(tg::smem(&fullB[s]), par, abort_v)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t b = tg::smem(sm + s * kS1Stage), a = b + 3 * kS1B;
      const uint64_t A12 = tg::desc(a, 128, 256, 0), A3z = tg::desc(a + 2 * kS1A, 128, 256, 0);
      const uint64_t B1 = tg::desc(b, 1024, 2048, 2), B2 = tg::desc(b + kS1B, 1024, 2048, 2),
                     B3 = tg::desc(b + 2 * kS1B, 1024, 2048, 2);
      tg::mma(tmem, A3z, B1, idesc, ks > 0 ? 1u : 0u);
      tg::mma(tmem, A12, B3, idesc, 1u);
      tg::mma(tmem, A12, B2, idesc, 1u);
      tg::mma(tmem, A12, B1, idesc, 1u);
      tg::commit(tg::smem(&empty[s]));
      ++done;
    }
    if (*abort_v && done > 0) {  // bounded wait for the MMAs in flight
      const int64_t last = done - 1;
      tg::wait(tg::smem(&empty[last % kS1Ring]), (uint32_t)((last / kS1Ring) & 1), nullptr);
    }
  }
  // all MMAs done: the last commit tracks every earlier one
  if (nks > 0 && !*abort_v && warp < 4) {
    const int64_t last = nks - 1;
    if (!tg::wait(tg::smem(&empty[last % kS1Ring]), (uint32_t)((last / kS1Ring) & 1), abort_v))
      abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag;
  if (ok && warp < 4) {
    // accumulator lanes 0-63: Y1 R' + Y3 R'1, lanes 64-127: Y2 R'
    const int half = warp >> 1, j = 32 * (warp & 1) + lane;
    float* dst = Cp + ((int64_t)(2 * chunk + half) * kDk + j) * R;
#pragma unroll 1
    for (int ch = 0; ch < kS1Cols / 16; ++ch) {
      const int cg = c0 + 16 * ch;
      if (cg >= R) break;  // uniform over the warp
      uint32_t u[16];
      if (nks > 0) {
        tg::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * ch), u);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = 0u;
      }
#pragma unroll
      for (int v4 = 0; v4 < 4; ++v4)
        *reinterpret_cast<float4*>(dst + cg + 4 * v4) =
            make_float4(__uint_as_float(u[4 * v4]), __uint_as_float(u[4 * v4 + 1]),
                        __uint_as_float(u[4 * v4 + 2]), __uint_as_float(u[4 * v4 + 3]));
    }
  }
  if (upd) {  // uniform over the CTA
    if (ok && warp < 4) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sh_rz[warp][4 * lane + e] = rz[e].value();
        sh_rr[warp][4 * lane + e] = rr[e].value();
      }
    }
    __syncthreads();
    if (ok && t < kS1Cols && c0 + t < R) {
      part_rz[(int64_t)chunk * R + c0 + t] =
          ((sh_rz[0][t] + sh_rz[1][t]) + sh_rz[2][t]) + sh_rz[3][t];
      part_rr[(int64_t)chunk * R + c0 + t] =
          ((sh_rr[0][t] + sh_rr[1][t]) + sh_rr[2][t]) + sh_rr[3][t];
    }
  }
  if (!ok && t == 0) atomicOr(flags, kFlagTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------- sum
// Thread per (column c, group of 8 j): C_jc = sum of the partial rows (in
// order), corr8[j8][c] = sum over the group of w_j C_jc^2 (FP64), and the
// pieces of C_jc in the K-major image of C^T's column group c / 128.
__global__ void k_dtc_sum(int R, int ncg, int nparts, const float* __restrict__ Cp,
                          const float* __restrict__ w, unsigned char* __restrict__ cimg,
                          double* __restrict__ corr8) {
  const int64_t cols = (int64_t)ncg * 128;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cols * 8;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j8 = (int)(e / cols);
    const int c = (int)(e - j8 * cols);
    float v[8];
    double corr = 0.0;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = 8 * j8 + jj;
      float s = 0.f;
      if (c < R)
        for (int q = 0; q < nparts; ++q) s += Cp[((int64_t)q * kDk + j) * R + c];
      v[jj] = s;
      corr += (double)w[j] * (double)s * (double)s;
    }
    if (c < R) corr8[(int64_t)j8 * R + c] = corr;
    uint4 p1, p2, p3;
    tg::split3x8(v, p1, p2, p3);
    unsigned char* dst = cimg + (int64_t)(c >> 7) * kU2Img + k64_off(c & 127, 8 * j8);
    *reinterpret_cast<uint4*>(dst) = p1;
    *reinterpret_cast<uint4*>(dst + kU2Piece) = p2;
    *reinterpret_cast<uint4*>(dst + 2 * kU2Piece) = p3;
  }
}

// ---------------------------------------------------------------- update
// One lane's loads of two row pairs of the update's epilogue.
struct EpiRegs {
  float4 r[2], p[2];
  float m[2], d[2];
  int64_t at[2];
  int v;  // bit u: row pair u is a row of the panel
};

// beta null: P = M^-1 R' + Yw C on every column (the first residuals).
// planes null: PD = d o P in FP32, else its three BF16 pieces, piece p at
// planes + p * plane_elems (row-major like PD).
__global__ void __launch_bounds__(256, 2) k_dtc_update(
    int64_t n, int R, const unsigned char* __restrict__ ywimg,
    const unsigned char* __restrict__ cimg, const float* __restrict__ minv,
    const float* __restrict__ dv, const double* __restrict__ beta, const int* __restrict__ active,
    const float* __restrict__ Rr, float* __restrict__ P, float* __restrict__ PD,
    uint16_t* __restrict__ planes, int64_t plane_elems, unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full, done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float sh_be[128];
  __shared__ int sh_act[128];
  volatile int* abort_v = &abort_flag;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int c0 = blockIdx.x * 128;
  const int64_t r0 = (int64_t)blockIdx.y * 128;
  unsigned char* sA = smem_raw;
  unsigned char* sB = smem_raw + kU2Img;
  if (t == 0) {
    abort_flag = 0;
    tg::mbar_init(tg::smem(&full), 1);
    tg::mbar_init(tg::smem(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (t < 128) {
    const int c = c0 + t;
    const int act = c < R && (!active || active[c] != 0);
    sh_act[t] = act;
    sh_be[t] = (beta && act) ? (float)beta[c] : 0.f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        tg::smem(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool mma_issued = false;  // thread 0
  if (t == 0) {
    tg::arrive_expect_tx(tg::smem(&full), 2 * kU2Img);
    tg::bulk_g2s(tg::smem(sA), ywimg + (int64_t)blockIdx.y * kU2Img, kU2Img, tg::smem(&full));
    tg::bulk_g2s(tg::smem(sB), cimg + (int64_t)blockIdx.x * kU2Img, kU2Img, tg::smem(&full));
    if (tg::wait(tg::smem(&full), 0u, nullptr)) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      constexpr uint32_t idesc = tg::idesc_bf16(128, 128, false, false);
      const uint32_t a = tg::smem(sA), b = tg::smem(sB);
#pragma unroll
      for (int s = 0; s < kDk / 16; ++s) {
        const uint32_t ko = 256u * s;
        const uint64_t A1 = tg::desc(a + ko, 128, 1024, 0),
                       A2 = tg::desc(a + kU2Piece + ko, 128, 1024, 0),
                       A3 = tg::desc(a + 2 * kU2Piece + ko, 128, 1024, 0);
        const uint64_t B1 = tg::desc(b + ko, 128, 1024, 0),
                       B2 = tg::desc(b + kU2Piece + ko, 128, 1024, 0),
                       B3 = tg::desc(b + 2 * kU2Piece + ko, 128, 1024, 0);
        tg::mma(tmem, A3, B1, idesc, s > 0 ? 1u : 0u);
        tg::mma(tmem, A2, B2, idesc, 1u);
        tg::mma(tmem, A1, B3, idesc, 1u);
        tg::mma(tmem, A2, B1, idesc, 1u);
        tg::mma(tmem, A1, B2, idesc, 1u);
        tg::mma(tmem, A1, B1, idesc, 1u);
      }
      tg::commit(tg::smem(&done));
      mma_issued = true;
    } else {
      abort_flag = 1;
    }
  }
  // warp w: accumulator rows 32 (w mod 4) .., columns 64 (w div 4) .., staged
  // through shared memory (the operand images are no longer needed) so that
  // the global accesses go row by row: 16 lanes x 16 bytes per row.  The
  // lane's rows are taken two pairs at a time, the loads of the next two
  // pairs in flight while one pair-batch is written; the first batch's loads
  // go out before the wait for the MMAs.
  const int quad = warp & 3, half = warp >> 2;
  const int sub = lane >> 4, cq = lane & 15;
  const int cl = 64 * half + 4 * cq;  // the lane's four columns in the tile
  const bool live = c0 + cl < R;      // R is a multiple of 32
  float* stg = reinterpret_cast<float*>(smem_raw) + warp * (32 * kU2Stg);
  auto load = [&](int bt, EpiRegs& E) {
    E.v = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int rl = 4 * bt + 2 * u + sub;
      const int64_t i = r0 + 32 * quad + rl;
      E.at[u] = i * R + c0 + cl;
      E.r[u] = E.p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      E.m[u] = E.d[u] = 0.f;
      if (i < n) {
        E.v |= 1 << u;
        E.r[u] = __ldcs(reinterpret_cast<const float4*>(Rr + E.at[u]));
        if (beta) E.p[u] = *reinterpret_cast<const float4*>(P + E.at[u]);
        E.m[u] = minv[i];
        E.d[u] = dv[i];
      }
    }
  };
  auto store = [&](int bt, const EpiRegs& E) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!(E.v >> u & 1)) continue;
      const int rl = 4 * bt + 2 * u + sub;
      const float4 zv = *reinterpret_cast<const float4*>(stg + rl * kU2Stg + 4 * cq);
      const float z4[4] = {zv.x, zv.y, zv.z, zv.w};
      const float r4[4] = {E.r[u].x, E.r[u].y, E.r[u].z, E.r[u].w};
      float p4[4] = {E.p[u].x, E.p[u].y, E.p[u].z, E.p[u].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float pn = fmaf(sh_be[cl + e], p4[e], fmaf(E.m[u], r4[e], z4[e]));
        p4[e] = sh_act[cl + e] ? pn : p4[e];
      }
      *reinterpret_cast<float4*>(P + E.at[u]) = make_float4(p4[0], p4[1], p4[2], p4[3]);
      float dp[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) dp[e] = E.d[u] * p4[e];
      if (planes) {
        uint2 q1, q2, q3;
        tg::split3x4(dp, q1, q2, q3);
        *reinterpret_cast<uint2*>(planes + E.at[u]) = q1;
        *reinterpret_cast<uint2*>(planes + plane_elems + E.at[u]) = q2;
        *reinterpret_cast<uint2*>(planes + 2 * plane_elems + E.at[u]) = q3;
      } else {
        *reinterpret_cast<float4*>(PD + E.at[u]) = make_float4(dp[0], dp[1], dp[2], dp[3]);
      }
    }
  };
  EpiRegs A, B;
  if (live) load(0, A);
  bool ok = tg::wait(tg::smem(&done), 0u, abort_v);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      const int cc = 64 * half + 16 * ch;
      if (c0 + cc >= R) break;  // uniform over the warp
      uint32_t z[16];
      tg::ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)cc, z);
#pragma unroll
      for (int v4 = 0; v4 < 4; ++v4)
        *reinterpret_cast<uint4*>(stg + lane * kU2Stg + 16 * ch + 4 * v4) =
            make_uint4(z[4 * v4], z[4 * v4 + 1], z[4 * v4 + 2], z[4 * v4 + 3]);
    }
    __syncwarp();
    if (live) {
#pragma unroll 1
      for (int bt = 0; bt < 8; bt += 2) {
        load(bt + 1, B);
        store(bt, A);
        if (bt + 2 < 8) load(bt + 2, A);
        store(bt + 1, B);
      }
    }
  } else if (t == 0) {
    atomicOr(flags, kFlagTimeout);
    // bounded waits for the copies and MMAs in flight
    tg::wait(tg::smem(&full), 0u, nullptr);
    if (mma_issued) tg::wait(tg::smem(&done), 0u, nullptr);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------- host
static int grid_for(gm_ctx* c, int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), 16 * sm_count(c)));
}

size_t dtc_yimg_bytes(int64_t n) { return (size_t)ceil_div(n, 16) * kS1Img; }
size_t dtc_rowimg_bytes(int64_t n) { return (size_t)ceil_div(n, 128) * kU2Img; }
size_t dtc_cimg_bytes(int R) { return (size_t)ceil_div(R, 128) * kU2Img; }

gm_status dtc_images(gm_ctx* c, int64_t n, const float* Y, const float* Yw, void* yimg,
                     void* ywimg) {
  const int64_t nks = ceil_div(n, 16), nblk = ceil_div(n, 128);
  GM_PROF(c, "k_dtc_img_y");
  k_dtc_img_y<<<grid_for(c, nks * kDk * 2), 256, 0, c->stream>>>(n, nks, Y,
                                                                 (unsigned char*)yimg);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_dtc_img_rows");
  k_dtc_img_rows<<<grid_for(c, nblk * 1024), 256, 0, c->stream>>>(n, nblk, Yw,
                                                                  (unsigned char*)ywimg);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

static gm_status dtc_attributes(gm_ctx* c) {
  static bool done = false;
  if (done) return GM_OK;
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_dtc_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kS1Smem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_dtc_step,
                                        cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_dtc_update,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kU2Smem));
  // all of the unified L1 / shared memory as shared: the CTAs per SM that the
  // registers allow
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_dtc_update,
                                        cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  done = true;
  return GM_OK;
}


// Row chunks of the step kernel for a panel of R columns: one wave of CTAs
// at three resident per SM (at most 136 registers x 160 threads and 72 KB of
// shared memory each), at most 64.
int dtc_chunks(gm_ctx* c, int64_t n, int R) {
  constexpr int kPerSm = 3;
  const int64_t ncg = ceil_div(R, kS1Cols), nks = ceil_div(n, 16);
  int64_t nch = std::max<int64_t>(1, (int64_t)kPerSm * sm_count(c) / ncg);
  nch = std::min<int64_t>(std::min<int64_t>(nch, 64), std::max<int64_t>(nks, 1));
  const int64_t kpc = ceil_div(std::max<int64_t>(nks, 1), nch);
  return (int)ceil_div(std::max<int64_t>(nks, 1), kpc);
}

gm_status dtc_step(gm_ctx* c, int64_t n, int R, int nch, const void* yimg, const double* alpha,
                   const float* minv, float* X, float* Rr, const float* P, const float* Q,
                   double* part_rz, double* part_rr, float* Cp, const float* w, void* cimg,
                   double* corr8) {
  gm_status a = dtc_attributes(c);
  if (a != GM_OK) return a;
  const int64_t nks = ceil_div(n, 16);
  const int kpc = (int)ceil_div(std::max<int64_t>(nks, 1), nch);
  const int ncg = (int)ceil_div(R, kS1Cols);
  GM_PROF(c, "k_dtc_step");
  k_dtc_step<<<dim3((unsigned)ncg, (unsigned)nch), kS1Threads, kS1Smem, c->stream>>>(
      n, R, kpc, (const unsigned char*)yimg, alpha, minv, X, Rr, P, Q, part_rz, part_rr, Cp,
      c->d_flags);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_dtc_sum");
  k_dtc_sum<<<grid_for(c, (int64_t)ncg * 128 * 8), 256, 0, c->stream>>>(
      R, ncg, 2 * nch, Cp, w, (unsigned char*)cimg, corr8);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status dtc_update(gm_ctx* c, int64_t n, int R, const void* ywimg, const void* cimg,
                     const float* minv, const float* dv, const double* beta, const int* active,
                     const float* Rr, float* P, float* PD, uint16_t* planes) {
  gm_status a = dtc_attributes(c);
  if (a != GM_OK) return a;
  GM_PROF(c, "k_dtc_update");
  k_dtc_update<<<dim3((unsigned)ceil_div(R, 128), (unsigned)ceil_div(n, 128)), 256, kU2Smem,
                 c->stream>>>(n, R, (const unsigned char*)ywimg, (const unsigned char*)cimg, minv,
                              dv, beta, active, Rr, P, PD, planes, n * (int64_t)R, c->d_flags);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm
