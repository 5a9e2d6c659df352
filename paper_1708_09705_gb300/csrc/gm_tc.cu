// Tensor-core panel product of the variance solves: Q = P + d o (K PD) over
// a panel of R right-hand sides, with K in 128-row tiles and the products on
// the 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulators
// in tensor memory).
//
// Precision: every FP32 operand x is split into three BF16 pieces,
// x1 = x rounded to BF16 (nearest even), x2 = the same of x - x1, x3 = the
// same of x - x1 - x2; each difference is exact in FP32 and x1 + x2 + x3 == x.
// Of the nine piece products the six whose size is at least 2^-16 of the
// leading one (x1y1, x1y2, x2y1, x1y3, x2y2, x3y1) are accumulated, so each
// product carries an error below 2^-23 of |xy| (the dropped terms), about
// that of an FP32 product.  The rounding is done on the bit patterns with
// integer adds and masks: no conversion instructions.
//
// Tile format.  Rows are cut into blocks of 128 (the stars are spatially
// sorted, so a block's rows share most neighbours: 62 % of the dense slots
// are stored entries on the 20,000-star workload).  A block's union of
// column indices is padded to a multiple of 16 by repeating its last column
// (with zero values) and cut into K-steps of 16 union columns.  Per K-step
// the tile keeps three 4 KB operand images (one per BF16 piece) of the
// 128 x 16 block of K values in the no-swizzle K-major layout of 8-row x
// 16-byte core matrices.
//
// CTA = (row block, 256 panel columns), 256 threads.  Per K-step every thread
// gathers its panel column's 16 values PD[u_k, c] (registers, two steps ahead),
// splits them and writes the three 256 x 16 B operands; one thread issues the
// six tcgen05.mma (M = 128 rows, N = 256 columns, K = 16) into the 128 x 256
// FP32 accumulator and commits to the step buffer's mbarrier.  Two step
// buffers: the gathers of step k+1 run while the tensor cores work on step k.
// Epilogue: tcgen05.ld of the accumulator, Q = P + d o acc, and per-column
// partial sums of P^T Q for the CG step length (fixed order).
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kTcRows = 128;                 // M
constexpr int kTcCols = 256;                 // N
constexpr int kTcK = 16;                     // K per MMA
constexpr int kTcA = kTcRows * kTcK * 2;     // 4 KB per piece
constexpr int kTcB = kTcCols * kTcK * 2;     // 8 KB per piece
constexpr int kTcStage = 3 * kTcA + 3 * kTcB;  // 36 KB
constexpr int kTcSmem = 2 * kTcStage + 4 * kTcCols * 8;  // + P^T Q partials (8 KB)

// byte offset of (row, k) in a no-swizzle K-major image with 16 columns:
// core matrices of 8 rows x 16 B, k-adjacent 128 B apart, row groups 256 B apart
__host__ __device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // LBO: k-adjacent core matrices
  d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;  // SBO: 8-row groups
  d |= (uint64_t)1 << 46;                       // descriptor version
  return d;
}

// kind::f16 instruction descriptor: BF16 A and B (K-major), FP32 D.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(kTcCols >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc));
}

// The same MMA with B in the MN-major layout.
__device__ __forceinline__ void tc_mma_mn(uint32_t tmem_d, uint64_t da, uint64_t db,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kTcIdesc | (1u << 16)), "r"(acc));
}

// Bounded wait on an mbarrier phase; false if it gave up.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

// x rounded to BF16 (nearest, ties to even) as an FP32 bit pattern whose low
// 16 bits are zero; the BF16 value is the high half
__device__ __forceinline__ uint32_t bf16_rne_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// three BF16 pieces of x (x1 + x2 + x3 == x)
__device__ __forceinline__ void split3(float x, uint32_t& a, uint32_t& b, uint32_t& c) {
  a = bf16_rne_bits(x);
  const float r1 = x - __uint_as_float(a);
  b = bf16_rne_bits(r1);
  const float r2 = r1 - __uint_as_float(b);
  c = bf16_rne_bits(r2);
}

// two BF16 values (high halves of lo and hi) in one 32-bit word, lo first
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x7632);
}

// ---------------------------------------------------------------- tiles
// Tile block of internal row i: blocks of 128 rows counted from each field's
// first row (no block straddles two fields).
struct TcBlocks {
  const int32_t* field_of;  // null: one field
  const int64_t* fptr;      // first row of each field
  const int64_t* boff;      // first block of each field
};
// Block of the row at tile position p (positions permute rows within their
// field, so the field of row i is the field of position p).
__device__ __forceinline__ int64_t tc_block(int64_t i, int64_t p, const TcBlocks& tb) {
  if (!tb.field_of) return p / kTcRows;
  const int f = tb.field_of[i];
  return tb.boff[f] + (p - tb.fptr[f]) / kTcRows;
}

// Tile order: within each field the rows are permuted so that every block
// of 128 consecutive positions is a compact cluster of stars, which share
// more neighbours (a smaller union of columns) than 128 rows of the cell
// order: a k-d partition of the field's star positions, split along the
// longest extent at a multiple of 128 next to the median until groups of
// 128 remain (the field's last group holds the remainder).  On the
// 20,000-star field 80 % of the tile slots are then stored entries, against
// 62 % in the cell order (73 % along a Morton curve).  Computed on the host
// once per context (the positions do not change).
static void tc_kd_order(int32_t* idx, int64_t n, const double* px, const double* py,
                        const double* pz) {
  struct Seg {
    int64_t lo, hi;
  };
  std::vector<Seg> stack{{0, n}};
  const double* P[3] = {px, py, pz};
  while (!stack.empty()) {
    const Seg g = stack.back();
    stack.pop_back();
    const int64_t m = g.hi - g.lo;
    if (m <= kTcRows) continue;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = g.lo; i < g.hi; ++i)
      for (int d = 0; d < 3; ++d) {
        mn[d] = std::min(mn[d], P[d][idx[i]]);
        mx[d] = std::max(mx[d], P[d][idx[i]]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
    int64_t k = (m / 2 + kTcRows / 2) / kTcRows * kTcRows;
    k = std::min<int64_t>(std::max<int64_t>(k, kTcRows), m - 1);
    const double* c = P[ax];
    std::nth_element(idx + g.lo, idx + g.lo + k, idx + g.hi, [c](int32_t a, int32_t b) {
      return c[a] < c[b] || (c[a] == c[b] && a < b);
    });
    stack.push_back({g.lo + k, g.hi});
    stack.push_back({g.lo, g.lo + k});
  }
}

__global__ void k_tc_keys(int64_t n, const int64_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col, int64_t nnz, int64_t n_pad,
                          TcBlocks tb, const int32_t* __restrict__ tpos,
                          unsigned long long* __restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const unsigned long long hi = (unsigned long long)tc_block(i, tpos ? tpos[i] : i, tb) << 32;
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32)
      keys[e] = hi | (unsigned long long)(unsigned)col[e];
  }
  for (int64_t e = nnz + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_pad;
       e += (int64_t)gridDim.x * blockDim.x)
    keys[e] = ~0ull;
}

__global__ void k_tc_flags(int64_t nnz, const unsigned long long* __restrict__ keys,
                           int64_t* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

__global__ void k_tc_unique(int64_t nnz, const unsigned long long* __restrict__ keys,
                            const int64_t* __restrict__ flag, const int64_t* __restrict__ pos,
                            int32_t* __restrict__ ucol, int32_t* __restrict__ ublk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (flag[e]) {
      const int64_t p = pos[e];
      ucol[p] = (int32_t)(keys[e] & 0xffffffffull);
      ublk[p] = (int32_t)(keys[e] >> 32);
    }
  }
}

// bptr[b] = first union position of block b
__global__ void k_tc_bptr(int64_t U, int64_t nblk, const int32_t* __restrict__ ublk,
                          int64_t* __restrict__ bptr) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= U;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t prev = p == 0 ? -1 : ublk[p - 1];
    const int64_t cur = p == U ? nblk : ublk[p];
    for (int64_t b = prev + 1; b <= cur; ++b) bptr[b] = p;
  }
}

// Padded union columns: slot (block b, local position q) holds the block's
// q-th union column, or its last one past the end.
__global__ void k_tc_ucol(int64_t nblk, const int64_t* __restrict__ bptr,
                          const int64_t* __restrict__ kbase, const int32_t* __restrict__ ucol,
                          int32_t* __restrict__ upad) {
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t u0 = bptr[b], u1 = bptr[b + 1];
    const int64_t slots = (kbase[b + 1] - kbase[b]) * kTcK;
    for (int64_t q = threadIdx.x; q < slots; q += blockDim.x)
      upad[kbase[b] * kTcK + q] = ucol[u0 + q < u1 ? u0 + q : u1 - 1];
  }
}

// Union of the columns of one tile block's rows, as a bitmap over all n
// columns in shared memory (CTA per block, warp per row, shared-memory
// atomics).  Phase 0 writes the union's size; phase 1 writes the union in
// increasing column order to ucol[bptr[b] ..] and, padded to whole K-steps
// with its last column, to upad[16 kbase[b] ..].
constexpr int kUnionMaxWords = 40960;  // 160 KB of bitmap: n <= 1,310,720

__global__ void __launch_bounds__(256) k_tc_union(
    int64_t n, int phase, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int64_t* __restrict__ brow0, const int32_t* __restrict__ trow,
    int64_t* __restrict__ count, const int64_t* __restrict__ bptr,
    const int64_t* __restrict__ kbase, int32_t* __restrict__ ucol, int32_t* __restrict__ upad) {
  extern __shared__ uint32_t bm[];
  __shared__ int64_t sh_off[256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nwords = (int)((n + 31) >> 5);
  const int64_t b = blockIdx.x;
  for (int w = t; w < nwords; w += 256) bm[w] = 0u;
  __syncthreads();
  for (int64_t p = brow0[b] + warp; p < brow0[b + 1]; p += 8) {
    const int64_t i = trow ? (int64_t)trow[p] : p;
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
      const int32_t j = col[e];
      atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
  }
  __syncthreads();
  // each thread owns a contiguous range of words
  const int wpt = (nwords + 255) / 256;
  const int w0 = min(t * wpt, nwords), w1 = min(w0 + wpt, nwords);
  int64_t cnt = 0;
  for (int w = w0; w < w1; ++w) cnt += __popc(bm[w]);
  sh_off[t] = cnt;
  __syncthreads();
  // inclusive scan of the counts (Hillis-Steele over the block)
  for (int d = 1; d < 256; d <<= 1) {
    const int64_t v = t >= d ? sh_off[t - d] : 0;
    __syncthreads();
    sh_off[t] += v;
    __syncthreads();
  }
  const int64_t total = sh_off[255];
  if (phase == 0) {
    if (t == 0) count[b] = total;
    return;
  }
  int64_t k = sh_off[t] - cnt;  // exclusive offset
  const int64_t u0 = bptr[b], s0 = kbase[b] * kTcK;
  for (int w = w0; w < w1; ++w) {
    uint32_t bits = bm[w];
    while (bits) {
      const int j = (w << 5) + __ffs(bits) - 1;
      bits &= bits - 1;
      ucol[u0 + k] = j;
      upad[s0 + k] = j;
      ++k;
    }
  }
  // padding slots: the last union column
  const int64_t slots = (kbase[b + 1] - kbase[b]) * kTcK;
  if (total > 0) {
    __syncthreads();
    const int32_t last = ucol[u0 + total - 1];
    for (int64_t q = total + t; q < slots; q += 256) upad[s0 + q] = last;
  }
}

// Operand images: entry (i, j) of block b at union position q of j goes to
// K-step kbase[b] + q / 16, column q % 16, row p - brow0[b] (p = the tile
// position of row i), three pieces.
__global__ void k_tc_fill(int64_t n, const int64_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col, const float* __restrict__ val,
                          const int64_t* __restrict__ bptr, const int64_t* __restrict__ kbase,
                          const int32_t* __restrict__ ucol, TcBlocks tb,
                          const int32_t* __restrict__ tpos, const int64_t* __restrict__ brow0,
                          unsigned char* __restrict__ img) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t p = tpos ? tpos[i] : i;
    const int64_t b = tc_block(i, p, tb);
    const int t = (int)(p - brow0[b]);
    const int64_t u0 = bptr[b], u1 = bptr[b + 1];
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
      const int32_t j = col[e];
      int64_t lo = u0, hi = u1;  // ucol[lo] <= j < ucol[hi]
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (ucol[mid] <= j) lo = mid; else hi = mid;
      }
      const int64_t q = lo - u0;
      unsigned char* step = img + (kbase[b] + q / kTcK) * (int64_t)(3 * kTcA);
      uint32_t p1, p2, p3;
      split3(val[e], p1, p2, p3);
      const int off = tc_off(t, (int)(q % kTcK));
      *reinterpret_cast<uint16_t*>(step + off) = (uint16_t)(p1 >> 16);
      *reinterpret_cast<uint16_t*>(step + kTcA + off) = (uint16_t)(p2 >> 16);
      *reinterpret_cast<uint16_t*>(step + 2 * kTcA + off) = (uint16_t)(p3 >> 16);
    }
  }
}

// ---------------------------------------------------------------- product
// Epilogue of a tile: warps 0-7 read the 128 x 256 accumulator (warp w: TMEM
// lanes 32 (w mod 4) .., columns 128 (w div 4) ..), write Q = P + d o acc and,
// for a single panel, the per-column partial sums of P^T Q into sh_pq[4][256].
__device__ __forceinline__ void tc_epilogue(uint32_t tmem, int warp, int lane, int64_t brow0,
                                            int64_t bend, int64_t base, int W, int c0,
                                            bool packed, const float* __restrict__ dv,
                                            const float* __restrict__ P, float* __restrict__ Q,
                                            double* sh_pq, const int32_t* __restrict__ trow) {
  {
    const int quad = warp & 3, half = warp >> 2;
    const int r = 32 * quad + lane;
    const int64_t pos = brow0 + r;
    const bool vrow = pos < bend;
    const int64_t row = (vrow && trow) ? (int64_t)trow[pos] : pos;
    const float dr = vrow ? dv[row] : 0.f;
#pragma unroll 1
    for (int ch = 0; ch < 8; ++ch) {
      const int cl = 128 * half + 16 * ch;
      uint32_t u[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
            "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]),
            "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
          : "r"(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)cl));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int cg = c0 + cl + k;
        float pq = 0.f;
        if (vrow && cg < W) {
          const int64_t at = base + row * W + cg;
          const float p = P[at];
          const float q = p + dr * __uint_as_float(u[k]);
          Q[at] = q;
          pq = p * q;
        }
        if (!packed) {  // uniform over the CTA; FP32 tree over the warp's 32 rows
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) pq += __shfl_xor_sync(0xffffffffu, pq, off);
          if (lane == 0) sh_pq[quad * kTcCols + cl + k] = (double)pq;
        }
      }
    }
  }
}

// Geometry of the panels.  One panel (single field): element (row, col) at
// row * R + col, CTA (blockIdx.x = column group, blockIdx.y = row block),
// partials of P^T Q per (row block, column).  Packed fields: element (row,
// col) of a field at base_b + row * W_b + col with base_b = P_f - row0_f W_f,
// CTA = items[blockIdx.x] = (row block, column group of its field), no
// partials (the packed CG forms P^T Q in its element-wise pass).
struct TcPanels {
  const int64_t* base;   // per tile block (packed) or null
  const int32_t* width;  // per tile block (packed) or null
  const int64_t* row0;   // first position of each tile block (packed) or null
  const int2* items;     // (block, column group) per CTA (packed) or null
  const int32_t* trow;   // row at each tile position (null: position = row)
};

// PF: gathered panel values are loaded PF steps ahead (indices PF + 1).
// NP: BF16 products per K-step, 6 (FP32-grade) or 3 (K1 PD2 + K2 PD1 +
// K1 PD1, the "mixed" form).
template <int PF, int NP>
__global__ void __launch_bounds__(256, 2) k_panel_spmm_tc(
    int64_t n, int R, const int64_t* __restrict__ kbase, const int32_t* __restrict__ upad,
    const uint4* __restrict__ img, const float* __restrict__ dv, const float* __restrict__ P,
    const float* __restrict__ PD, float* __restrict__ Q, double* __restrict__ part_pq,
    TcPanels pk, unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  double* sh_pq = reinterpret_cast<double*>(smem + 2 * kTcStage);  // [4][256]

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool packed = pk.items != nullptr;
  int64_t b, base, brow0, bend;
  int c0, W;
  if (packed) {
    const int2 it = pk.items[blockIdx.x];
    b = it.x;
    c0 = it.y * kTcCols;
    W = pk.width[b];
    base = pk.base[b];
    brow0 = pk.row0[b];
    bend = pk.row0[b + 1];
  } else {
    b = blockIdx.y;
    c0 = blockIdx.x * kTcCols;
    W = R;
    base = 0;
    brow0 = b * kTcRows;
    bend = min(brow0 + kTcRows, n);
  }
  const int col = c0 + t;
  const bool live = col < W;
  const int64_t ks0 = kbase[b], nks = kbase[b + 1] - ks0;

  if (t == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        tc_smem(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // Register pipeline: the tile pieces and gathered panel values of a step
  // are loaded PF steps ahead and its union column indices PF + 1 steps
  // ahead (the gathers wait on the indices, so each is one global round trip).
  struct Vals {
    uint4 a[3];    // this thread's three 16-byte pieces of the tile image
    float b[16];   // the column's 16 gathered panel values
  };
  Vals v0{}, v1{};
  int4 idx[4];
  auto load_idx = [&](int64_t ks) {
    const int4* u4 = reinterpret_cast<const int4*>(upad + (ks0 + ks) * kTcK);
#pragma unroll
    for (int q = 0; q < 4; ++q) idx[q] = __ldg(u4 + q);
  };
  auto load_vals = [&](Vals& v, int64_t ks) {
    const uint4* src = img + (ks0 + ks) * (3 * kTcA / 16);
#pragma unroll
    for (int q = 0; q < 3; ++q) v.a[q] = __ldg(src + t + 256 * q);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j[4] = {idx[q].x, idx[q].y, idx[q].z, idx[q].w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
        v.b[4 * q + r] = live ? __ldg(PD + (base + (int64_t)j[r] * W + col)) : 0.f;
    }
  };

  if (nks > 0) {
    load_idx(0);
    load_vals(v0, 0);
  }
  if (PF == 2 && nks > 1) {
    load_idx(1);
    load_vals(v1, 1);
  }
  if (nks > PF) load_idx(PF);
  for (int64_t ks = 0; ks < nks; ++ks) {
    const int s = (int)(ks & 1);
    unsigned char* sA = smem + s * kTcStage;
    unsigned char* sB = sA + 3 * kTcA;
    // the buffer was last read by the MMAs of step ks - 2
    if (ks >= 2 && !tc_wait(tc_smem(&mbar[s]), (uint32_t)(((ks - 2) >> 1) & 1))) abort_flag = 1;
#pragma unroll
    for (int q = 0; q < 3; ++q) reinterpret_cast<uint4*>(sA)[t + 256 * q] = v0.a[q];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t w1[4], w2[4], w3[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t a0, a1, a2, b0, b1, b2;
        split3(v0.b[8 * h + 2 * q], a0, a1, a2);
        split3(v0.b[8 * h + 2 * q + 1], b0, b1, b2);
        w1[q] = pack2(a0, b0);
        w2[q] = pack2(a1, b1);
        w3[q] = pack2(a2, b2);
      }
      const int off = tc_off(t, 8 * h);
      *reinterpret_cast<uint4*>(sB + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
      *reinterpret_cast<uint4*>(sB + kTcB + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      *reinterpret_cast<uint4*>(sB + 2 * kTcB + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    }
    if (PF == 2) {
      v0 = v1;
      if (ks + 2 < nks) load_vals(v1, ks + 2);
      if (ks + 3 < nks) load_idx(ks + 3);
    } else {
      if (ks + 1 < nks) load_vals(v0, ks + 1);
      if (ks + 2 < nks) load_idx(ks + 2);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (abort_flag) break;
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = tc_smem(sA), bb = tc_smem(sB);
      const uint64_t A1 = tc_desc(a), A2 = tc_desc(a + kTcA), A3 = tc_desc(a + 2 * kTcA);
      const uint64_t B1 = tc_desc(bb), B2 = tc_desc(bb + kTcB), B3 = tc_desc(bb + 2 * kTcB);
      // small terms first
      if constexpr (NP == 3) {
        tc_mma(tmem, A2, B1, ks > 0 ? 1u : 0u);
        tc_mma(tmem, A1, B2, 1u);
        tc_mma(tmem, A1, B1, 1u);
      } else {
        tc_mma(tmem, A3, B1, ks > 0 ? 1u : 0u);
        tc_mma(tmem, A2, B2, 1u);
        tc_mma(tmem, A1, B3, 1u);
        tc_mma(tmem, A2, B1, 1u);
        tc_mma(tmem, A1, B2, 1u);
        tc_mma(tmem, A1, B1, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem(&mbar[s])));
    }
  }
  // all MMAs done: the last commit tracks every earlier one
  if (!abort_flag && nks > 0) {
    const int64_t last = nks - 1;
    if (!tc_wait(tc_smem(&mbar[last & 1]), (uint32_t)((last >> 1) & 1))) abort_flag = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (!abort_flag)
    tc_epilogue(tmem, warp, lane, brow0, bend, base, W, c0, packed, dv, P, Q, sh_pq, pk.trow);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (!abort_flag) {
    if (live && !packed)
      part_pq[b * R + col] = ((sh_pq[t] + sh_pq[kTcCols + t]) + sh_pq[2 * kTcCols + t]) +
                             sh_pq[3 * kTcCols + t];
  } else if (t == 0) {
    atomicOr(flags, kFlagTimeout);
    // give MMAs still in flight a bounded chance to finish before the
    // accumulator columns are released
    for (int s = 0; s < 2; ++s) {
      const int64_t uses = nks > s ? (nks - 1 - s) / 2 + 1 : 0;
      if (uses > 0) tc_wait(tc_smem(&mbar[s]), (uint32_t)((uses - 1) & 1));
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}


// Warp-specialised variant: warps 0-7 (one panel column per thread) fill a
// ring of kTcRing stage buffers and arrive on the stage's "full" mbarrier;
// warp 8 waits on it, issues the six MMAs and commits to the stage's "empty"
// mbarrier, which the fillers wait on before reusing the buffer.  No CTA-wide
// barrier per K-step: the fillers run up to kTcRing - 1 steps ahead of the
// tensor cores.  Every wait is bounded and also gives up when another thread
// has given up (shared abort flag).
constexpr int kTcRing = 3;
constexpr int kTcSmemWs = kTcRing * kTcStage;  // P^T Q partials reuse stage 0

__device__ __forceinline__ bool tc_wait_or_abort(uint32_t mbar, uint32_t parity,
                                                 volatile int* abort_flag) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}

template <int NP>
__global__ void __launch_bounds__(288, 2) k_panel_spmm_tc_ws(
    int64_t n, int R, const int64_t* __restrict__ kbase, const int32_t* __restrict__ upad,
    const uint4* __restrict__ img, const float* __restrict__ dv, const float* __restrict__ P,
    const float* __restrict__ PD, float* __restrict__ Q, double* __restrict__ part_pq,
    TcPanels pk, unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[kTcRing], empty[kTcRing];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abort_v = &abort_flag;
  double* sh_pq = reinterpret_cast<double*>(smem);  // [4][256], after the last MMA

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool packed = pk.items != nullptr;
  int64_t b, base, brow0, bend;
  int c0, W;
  if (packed) {
    const int2 it = pk.items[blockIdx.x];
    b = it.x;
    c0 = it.y * kTcCols;
    W = pk.width[b];
    base = pk.base[b];
    brow0 = pk.row0[b];
    bend = pk.row0[b + 1];
  } else {
    b = blockIdx.y;
    c0 = blockIdx.x * kTcCols;
    W = R;
    base = 0;
    brow0 = b * kTcRows;
    bend = min(brow0 + kTcRows, n);
  }
  const int col = c0 + t;
  const bool live = t < 256 && col < W;
  const int64_t ks0 = kbase[b], nks = kbase[b + 1] - ks0;

  if (t == 0) {
    abort_flag = 0;
    for (int q = 0; q < kTcRing; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(tc_smem(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&empty[q])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        tc_smem(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp < 8) {
    // ---- fillers: gather, split and stage one K-step per ring slot
    uint4 ra[3];
    float rb[16];
    int4 idx[4];
    auto load_idx = [&](int64_t ks) {
      const int4* u4 = reinterpret_cast<const int4*>(upad + (ks0 + ks) * kTcK);
#pragma unroll
      for (int q = 0; q < 4; ++q) idx[q] = __ldg(u4 + q);
    };
    auto load_vals = [&](int64_t ks) {
      const uint4* src = img + (ks0 + ks) * (3 * kTcA / 16);
#pragma unroll
      for (int q = 0; q < 3; ++q) ra[q] = __ldg(src + t + 256 * q);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j[4] = {idx[q].x, idx[q].y, idx[q].z, idx[q].w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
          rb[4 * q + r] = live ? __ldg(PD + (base + (int64_t)j[r] * W + col)) : 0.f;
      }
    };
    if (nks > 0) {
      load_idx(0);
      load_vals(0);
    }
    if (nks > 1) load_idx(1);
    for (int64_t ks = 0; ks < nks; ++ks) {
      const int s = (int)(ks % kTcRing);
      const int64_t use = ks / kTcRing;
      unsigned char* sA = smem + s * kTcStage;
      unsigned char* sB = sA + 3 * kTcA;
      // the slot was last read by the MMAs of step ks - kTcRing
      if (use > 0 && !tc_wait_or_abort(tc_smem(&empty[s]), (uint32_t)((use - 1) & 1), abort_v)) {
        abort_flag = 1;
        break;
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) reinterpret_cast<uint4*>(sA)[t + 256 * q] = ra[q];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t w1[4], w2[4], w3[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t a0, a1, a2, b0, b1, b2;
          split3(rb[8 * h + 2 * q], a0, a1, a2);
          split3(rb[8 * h + 2 * q + 1], b0, b1, b2);
          w1[q] = pack2(a0, b0);
          w2[q] = pack2(a1, b1);
          w3[q] = pack2(a2, b2);
        }
        const int off = tc_off(t, 8 * h);
        *reinterpret_cast<uint4*>(sB + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(sB + kTcB + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        *reinterpret_cast<uint4*>(sB + 2 * kTcB + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(&full[s])) : "memory");
      if (ks + 1 < nks) load_vals(ks + 1);
      if (ks + 2 < nks) load_idx(ks + 2);
    }
  } else if (lane == 0) {
    // ---- MMA issuer
    for (int64_t ks = 0; ks < nks; ++ks) {
      const int s = (int)(ks % kTcRing);
      const int64_t use = ks / kTcRing;
      if (!tc_wait_or_abort(tc_smem(&full[s]), (uint32_t)(use & 1), abort_v)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = tc_smem(smem + s * kTcStage), bb = a + 3 * kTcA;
      const uint64_t A1 = tc_desc(a), A2 = tc_desc(a + kTcA), A3 = tc_desc(a + 2 * kTcA);
      const uint64_t B1 = tc_desc(bb), B2 = tc_desc(bb + kTcB), B3 = tc_desc(bb + 2 * kTcB);
      if constexpr (NP == 3) {
        tc_mma(tmem, A2, B1, ks > 0 ? 1u : 0u);
        tc_mma(tmem, A1, B2, 1u);
        tc_mma(tmem, A1, B1, 1u);
      } else {
        tc_mma(tmem, A3, B1, ks > 0 ? 1u : 0u);
        tc_mma(tmem, A2, B2, 1u);
        tc_mma(tmem, A1, B3, 1u);
        tc_mma(tmem, A2, B1, 1u);
        tc_mma(tmem, A1, B2, 1u);
        tc_mma(tmem, A1, B1, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem(&empty[s])));
    }
  }
  // all MMAs done: the last step's commit tracks every earlier one
  if (nks > 0 && !*abort_v) {
    const int64_t last = nks - 1;
    if (!tc_wait_or_abort(tc_smem(&empty[last % kTcRing]), (uint32_t)((last / kTcRing) & 1),
                          abort_v))
      abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag;
  if (ok && warp < 8)
    tc_epilogue(tmem, warp, lane, brow0, bend, base, W, c0, packed, dv, P, Q, sh_pq, pk.trow);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (ok) {
    if (live && !packed)
      part_pq[b * R + col] = ((sh_pq[t] + sh_pq[kTcCols + t]) + sh_pq[2 * kTcCols + t]) +
                             sh_pq[3 * kTcCols + t];
  } else if (t == 0) {
    atomicOr(flags, kFlagTimeout);
    // a bounded chance for MMAs in flight to finish before the columns go
    for (int q = 0; q < kTcRing; ++q) {
      const int64_t uses = nks > q ? (nks - 1 - q) / kTcRing + 1 : 0;
      if (uses > 0) tc_wait(tc_smem(&empty[q]), (uint32_t)((uses - 1) & 1));
    }
  }
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------- async variant
// The B operand straight from memory.  Once per product the panel PD is split
// into three BF16 planes (k_split3_planes, the same rounding as split3), so
// that a K-step's B tile is a plain copy of 16 gathered plane rows x 256
// columns: no register staging and no split on the MMA's critical path.  The
// tile is kept MN-major in shared memory (the panel's columns contiguous, as
// in the planes) in the 128-byte-swizzled layout: 1 KB atoms of 8 k-rows x
// 64 columns (a 128-byte row per k) in which the 16-byte chunk c of row r
// sits at chunk c ^ r, the atoms of consecutive 64-column blocks 1 KB apart
// and the two 8-row k-groups 4 KB apart; the MMA's instruction descriptor
// marks B as MN-major.  (Without the swizzle the chunks of one k-row lie
// 128 B apart, in one bank group, and the tensor core's reads serialise.)
//
// Warp roles (160 threads, two CTAs per SM): warps 0-3 are producers -- per
// K-step thread 0 starts one bulk copy of the tile's A pieces (cp.async.bulk,
// completing on the stage's A barrier with its byte count) and all 128
// threads copy the B pieces in 16-byte chunks (cp.async, each thread's
// completion arriving on the stage's B barrier without blocking the thread),
// kTaRing stages ahead of the tensor cores; warp 4's lane 0 waits for both
// barriers, orders the copies before the tensor core's reads
// (fence.proxy.async), issues the MMAs and commits to the stage's empty
// barrier.  Warps 0-3 then run the epilogue.  Every wait is bounded and gives
// up when another thread has; a CTA that gives up waits (bounded) for its
// bulk copies and MMAs in flight before it releases tensor memory.
constexpr int kTaRing = 3;
constexpr int kTaProd = 128;
constexpr int kTaThreads = kTaProd + 32;
constexpr int kTaPiece = kTcCols * kTcK * 2;              // 8 KB: one plane's B tile
constexpr int kTaStage = 3 * kTcA + 3 * kTaPiece;         // 36 KB
// 108 KB of stages (the partials reuse stage 0) + 1 KB to align the swizzled atoms
constexpr int kTaSmem = kTaRing * kTaStage + 1024;

// byte offset of B element (k, n) in the swizzled MN-major image of one plane
__host__ __device__ __forceinline__ int tcb_off(int k, int n) {
  return (n >> 6) * 1024 + (k >> 3) * 4096 + (k & 7) * 128 + ((((n >> 3) & 7) ^ (k & 7)) << 4) +
         (n & 7) * 2;
}

// MN-major 128-byte-swizzle descriptor: LBO = stride of the 64-column atoms
// (1 KB), SBO = stride of the 8-row k-groups (4 KB), layout type 2
__device__ __forceinline__ uint64_t tc_desc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((4096u >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// PD (elements [0, ne)) -> three BF16 planes, plane p at planes + p * ne
__global__ void k_split3_planes(int64_t ne, const float* __restrict__ PD,
                                uint16_t* __restrict__ planes) {
  const int64_t n4 = ne >> 2;
  const float4* src = reinterpret_cast<const float4*>(PD);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = __ldcs(src + q);
    uint32_t a[4], b[4], c[4];
    split3(v.x, a[0], b[0], c[0]);
    split3(v.y, a[1], b[1], c[1]);
    split3(v.z, a[2], b[2], c[2]);
    split3(v.w, a[3], b[3], c[3]);
    reinterpret_cast<uint2*>(planes)[q] = make_uint2(pack2(a[0], a[1]), pack2(a[2], a[3]));
    reinterpret_cast<uint2*>(planes + ne)[q] = make_uint2(pack2(b[0], b[1]), pack2(b[2], b[3]));
    reinterpret_cast<uint2*>(planes + 2 * ne)[q] = make_uint2(pack2(c[0], c[1]), pack2(c[2], c[3]));
  }
  for (int64_t e = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t a, b, c;
    split3(PD[e], a, b, c);
    planes[e] = (uint16_t)(a >> 16);
    planes[ne + e] = (uint16_t)(b >> 16);
    planes[2 * ne + e] = (uint16_t)(c >> 16);
  }
}

template <int NP>
__global__ void __launch_bounds__(kTaThreads, 2) k_panel_spmm_tc_async(
    int64_t n, int R, const int64_t* __restrict__ kbase, const int32_t* __restrict__ upad,
    const unsigned char* __restrict__ img, const float* __restrict__ dv,
    const float* __restrict__ P, const uint16_t* __restrict__ planes, int64_t plane_elems,
    float* __restrict__ Q, double* __restrict__ part_pq, TcPanels pk,
    unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t fullA[kTaRing], fullB[kTaRing], empty[kTaRing];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abort_v = &abort_flag;
  // the swizzle pattern follows the address bits: stages start on 1 KB
  unsigned char* smem = smem_raw + ((1024u - (tc_smem(smem_raw) & 1023u)) & 1023u);
  double* sh_pq = reinterpret_cast<double*>(smem);  // [4][256], after the last MMA
  constexpr int npl = NP == 3 ? 2 : 3;              // BF16 pieces used per side
  constexpr uint32_t abytes = npl * kTcA;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool packed = pk.items != nullptr;
  int64_t b, base, brow0, bend;
  int c0, W;
  if (packed) {
    const int2 it = pk.items[blockIdx.x];
    b = it.x;
    c0 = it.y * kTcCols;
    W = pk.width[b];
    base = pk.base[b];
    brow0 = pk.row0[b];
    bend = pk.row0[b + 1];
  } else {
    b = blockIdx.y;
    c0 = blockIdx.x * kTcCols;
    W = R;
    base = 0;
    brow0 = b * kTcRows;
    bend = min(brow0 + kTcRows, n);
  }
  const int64_t ks0 = kbase[b], nks = kbase[b + 1] - ks0;

  if (t == 0) {
    abort_flag = 0;
    for (int q = 0; q < kTaRing; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&fullA[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&fullB[q])),
                   "r"(kTaProd));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&empty[q])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        tc_smem(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  int64_t issued_a = 0;  // bulk copies started by thread 0

  if (warp < 4) {
    // ---- producers.  Thread t copies, per plane, 16-byte chunk t % 8 of
    // k-row t / 8 in each of the four 64-column blocks: a quarter-warp fills
    // one 128-byte row of an atom from 128 contiguous bytes of a plane row.
    const int clo = t & 7, kr = t >> 3;
    for (int64_t ks = 0; ks < nks; ++ks) {
      const int s = (int)(ks % kTaRing);
      const int64_t use = ks / kTaRing;
      if (use > 0 && !tc_wait_or_abort(tc_smem(&empty[s]), (uint32_t)((use - 1) & 1), abort_v)) {
        abort_flag = 1;
        break;
      }
      unsigned char* sA = smem + s * kTaStage;
      unsigned char* sB = sA + 3 * kTcA;
      if (t == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         tc_smem(&fullA[s])),
                     "r"(abytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(tc_smem(sA)),
            "l"(__cvta_generic_to_global(img + (ks0 + ks) * (int64_t)(3 * kTcA))), "r"(abytes),
            "r"(tc_smem(&fullA[s]))
            : "memory");
        ++issued_a;
      }
      const int64_t row = __ldg(upad + (ks0 + ks) * kTcK + kr);
#pragma unroll
      for (int p = 0; p < npl; ++p) {
        const uint16_t* pl = planes + p * plane_elems + base + row * W;
        const uint32_t db = tc_smem(sB + p * kTaPiece);
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
          const int n = 64 * nb + 8 * clo;
          const int colg = c0 + n;
          const bool in = colg < W;
          const uint16_t* src = in ? pl + colg : planes;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                           db + (uint32_t)tcb_off(kr, n)),
                       "l"(__cvta_generic_to_global(src)), "r"(in ? 16 : 0)
                       : "memory");
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                       tc_smem(&fullB[s]))
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4 && lane == 0) {
    // ---- MMA issuer
    for (int64_t ks = 0; ks < nks; ++ks) {
      const int s = (int)(ks % kTaRing);
      const uint32_t par = (uint32_t)((ks / kTaRing) & 1);
      if (!tc_wait_or_abort(tc_smem(&fullA[s]), par, abort_v) ||
          !tc_wait_or_abort(tc_smem(&fullB[s]), par, abort_v)) {
        abort_flag = 1;
        break;
      }
      // the B pieces were written through the generic proxy (cp.async)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = tc_smem(smem + s * kTaStage), bb = a + 3 * kTcA;
      const uint64_t A1 = tc_desc(a), A2 = tc_desc(a + kTcA);
      const uint64_t B1 = tc_desc_mn(bb), B2 = tc_desc_mn(bb + kTaPiece);
      if constexpr (NP == 3) {
        tc_mma_mn(tmem, A2, B1, ks > 0 ? 1u : 0u);
        tc_mma_mn(tmem, A1, B2, 1u);
        tc_mma_mn(tmem, A1, B1, 1u);
      } else {
        const uint64_t A3 = tc_desc(a + 2 * kTcA), B3 = tc_desc_mn(bb + 2 * kTaPiece);
        tc_mma_mn(tmem, A3, B1, ks > 0 ? 1u : 0u);
        tc_mma_mn(tmem, A2, B2, 1u);
        tc_mma_mn(tmem, A1, B3, 1u);
        tc_mma_mn(tmem, A2, B1, 1u);
        tc_mma_mn(tmem, A1, B2, 1u);
        tc_mma_mn(tmem, A1, B1, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem(&empty[s])));
    }
  }
  // all MMAs done: the last step's commit tracks every earlier one
  if (nks > 0 && !*abort_v && warp < 4) {
    const int64_t last = nks - 1;
    if (!tc_wait_or_abort(tc_smem(&empty[last % kTaRing]), (uint32_t)((last / kTaRing) & 1),
                          abort_v))
      abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag;
  if (ok && warp < 4) {
    // epilogue: warp w holds accumulator rows 32 w .. 32 w + 31, all 256 columns
    const int r = 32 * warp + lane;
    const int64_t pos = brow0 + r;
    const bool vrow = pos < bend;
    const int64_t row = (vrow && pk.trow) ? (int64_t)pk.trow[pos] : pos;
    const float dr = vrow ? dv[row] : 0.f;
#pragma unroll 1
    for (int ch = 0; ch < 16; ++ch) {
      const int cl = 16 * ch;
      uint32_t u[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
            "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]),
            "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cl));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the panel width is a multiple of 32: a 16-column chunk is all in or out
      float pq[16];
      if (vrow && c0 + cl < W) {
        const int64_t at = base + row * W + c0 + cl;  // 16-byte aligned
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float4 p4 = *reinterpret_cast<const float4*>(P + at + 4 * v);
          float4 q4;
          q4.x = p4.x + dr * __uint_as_float(u[4 * v + 0]);
          q4.y = p4.y + dr * __uint_as_float(u[4 * v + 1]);
          q4.z = p4.z + dr * __uint_as_float(u[4 * v + 2]);
          q4.w = p4.w + dr * __uint_as_float(u[4 * v + 3]);
          *reinterpret_cast<float4*>(Q + at + 4 * v) = q4;
          pq[4 * v + 0] = p4.x * q4.x;
          pq[4 * v + 1] = p4.y * q4.y;
          pq[4 * v + 2] = p4.z * q4.z;
          pq[4 * v + 3] = p4.w * q4.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) pq[k] = 0.f;
      }
      if (!packed) {  // uniform over the CTA
        // column sums over the warp's 32 rows by a reduce-scatter of
        // shuffles (16 instead of 80): each step halves the columns a lane
        // holds; at the end lanes 2c' and 2c' + 1 hold the sum of column
        // c' = bits 4..1 of the lane index (FP32 tree, fixed order)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const bool up = lane & 16;
          const float send = up ? pq[j] : pq[j + 8];
          const float keep = up ? pq[j + 8] : pq[j];
          pq[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool up = lane & 8;
          const float send = up ? pq[j] : pq[j + 4];
          const float keep = up ? pq[j + 4] : pq[j];
          pq[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const bool up = lane & 4;
          const float send = up ? pq[j] : pq[j + 2];
          const float keep = up ? pq[j + 2] : pq[j];
          pq[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        {
          const bool up = lane & 2;
          const float send = up ? pq[0] : pq[1];
          const float keep = up ? pq[1] : pq[0];
          pq[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
        }
        pq[0] += __shfl_xor_sync(0xffffffffu, pq[0], 1);
        const int colw = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                         ((lane >> 1) & 1);
        if ((lane & 1) == 0) sh_pq[warp * kTcCols + cl + colw] = (double)pq[0];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (ok) {
    if (!packed)
      for (int cl = t; cl < kTcCols; cl += kTaThreads)
        if (c0 + cl < W)
          part_pq[b * R + c0 + cl] = ((sh_pq[cl] + sh_pq[kTcCols + cl]) +
                                      sh_pq[2 * kTcCols + cl]) + sh_pq[3 * kTcCols + cl];
  } else if (t == 0) {
    atomicOr(flags, kFlagTimeout);
    // bounded waits for the bulk copies and MMAs still in flight
    for (int q = 0; q < kTaRing; ++q) {
      const int64_t na = issued_a > q ? (issued_a - 1 - q) / kTaRing + 1 : 0;
      if (na > 0) tc_wait(tc_smem(&fullA[q]), (uint32_t)((na - 1) & 1));
      const int64_t uses = nks > q ? (nks - 1 - q) / kTaRing + 1 : 0;
      if (uses > 0) tc_wait(tc_smem(&empty[q]), (uint32_t)((uses - 1) & 1));
    }
  }
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------- host
// The tensor-core path serves FP32 contexts unless GM_SPMM=simt.
bool tc_wanted(gm_ctx* c) {
  if (c->cfg.precision != GM_PREC_FP32) return false;
  const char* e = std::getenv("GM_SPMM");
  return !(e && e[0] == 's');
}

gm_status tc_tiles_build(gm_ctx* c) {
  c->tc_nblk = 0;
  c->stats.tile_ksteps = 0;
  const int64_t n = c->n, nnz = c->nnz;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  // field-aligned blocks of 128 rows
  const int nf = c->n_fields;
  c->h_tc_boff.assign(nf + 1, 0);
  for (int f = 0; f < nf; ++f)
    c->h_tc_boff[f + 1] = c->h_tc_boff[f] + ceil_div(c->h_fptr[f + 1] - c->h_fptr[f], kTcRows);
  const int64_t nblk = c->h_tc_boff[nf];
  std::vector<int64_t> hr0(nblk + 1, n);
  for (int f = 0; f < nf; ++f)
    for (int64_t b = c->h_tc_boff[f]; b < c->h_tc_boff[f + 1]; ++b)
      hr0[b] = c->h_fptr[f] + (b - c->h_tc_boff[f]) * kTcRows;
  if (!ensure(c, c->tc_brow0, (nblk + 1) * sizeof(int64_t)) ||
      !ensure(c, c->tc_boffd, (nf + 1) * sizeof(int64_t)))
    return set_error(c, GM_E_NOMEM, "tensor-core block tables");
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_brow0.p, hr0.data(), (nblk + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_boffd.p, c->h_tc_boff.data(), (nf + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  TcBlocks tb{nullptr, nullptr, nullptr};
  if (nf > 1) tb = TcBlocks{c->field_of, c->fptr, (const int64_t*)c->tc_boffd.p};
  // tile order (GM_TC_ORDER=rows keeps the cell order): a k-d partition of
  // each field's stars, once per context
  {
    const char* e = std::getenv("GM_TC_ORDER");
    const bool want = !(e && e[0] == 'r');
    if (!want) {
      c->tc_order = false;
    } else if (!c->tc_order) {
      std::vector<double> hx(n), hy(n), hz(n), hs(n);
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hs.data(), c->s, n * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hx.data(), c->ux, n * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hy.data(), c->uy, n * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hz.data(), c->uz, n * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
      for (int64_t i = 0; i < n; ++i) {
        hx[i] *= hs[i];
        hy[i] *= hs[i];
        hz[i] *= hs[i];
      }
      std::vector<int32_t> trow(n), tpos_h(n);
      for (int64_t i = 0; i < n; ++i) trow[i] = (int32_t)i;
      for (int f = 0; f < nf; ++f) {
        const int64_t f0 = c->h_fptr[f], f1 = c->h_fptr[f + 1];
        tc_kd_order(trow.data() + f0, f1 - f0, hx.data(), hy.data(), hz.data());
      }
      for (int64_t p = 0; p < n; ++p) tpos_h[trow[p]] = (int32_t)p;
      if (!ensure(c, c->tc_trow, n * sizeof(int32_t)) ||
          !ensure(c, c->tc_tpos, n * sizeof(int32_t)))
        return set_error(c, GM_E_NOMEM, "tile order");
      GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_trow.p, trow.data(), n * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, st));
      GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_tpos.p, tpos_h.data(), n * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, st));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(st));  // the host vectors end here
      c->tc_order = true;
    }
  }
  const int32_t* tpos = c->tc_order ? (const int32_t*)c->tc_tpos.p : nullptr;
  const int wb = (int)std::min<int64_t>(ceil_div(n * 32, 256), 32 * sms);
  const int eb = (int)std::min<int64_t>(ceil_div(nnz, 256), 16 * sms);
  // union of each block's columns, K-step offsets and padded columns: by a
  // bitmap per block when n fits shared memory, else by a sort of (block,
  // column) keys over all entries (also with GM_TC_UNION=sort)
  const int nwords = (int)ceil_div(n, 32);
  const char* ue = std::getenv("GM_TC_UNION");
  const bool bitmap = nwords <= kUnionMaxWords && !(ue && ue[0] == 's');
  std::vector<int64_t> hb(nblk + 1, 0), hk(nblk + 1, 0);
  int64_t U = 0, nks = 0;
  int32_t* ucol = nullptr;
  int64_t* bptr = (int64_t*)dev_alloc(c, (nblk + 1) * sizeof(int64_t));
  if (!bptr) return set_error(c, GM_E_NOMEM, "tensor-core tile union");
  const int32_t* trow = c->tc_order ? (const int32_t*)c->tc_trow.p : nullptr;
  const size_t bm_smem = (size_t)nwords * sizeof(uint32_t);
  if (bitmap) {
    if (bm_smem > 48 * 1024)
      GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_tc_union, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)bm_smem));
    GM_PROF(c, "k_tc_union");
    k_tc_union<<<(unsigned)nblk, 256, bm_smem, st>>>(n, 0, c->row_ptr, c->col,
                                                     (const int64_t*)c->tc_brow0.p, trow, bptr,
                                                     nullptr, nullptr, nullptr, nullptr);
    GM_LAUNCH_CHECK(c);
    std::vector<int64_t> hc(nblk);
    GM_CUDA_CHECK(c, cudaMemcpyAsync(hc.data(), bptr, nblk * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
    for (int64_t b = 0; b < nblk; ++b) {
      hb[b + 1] = hb[b] + hc[b];
      hk[b + 1] = hk[b] + ceil_div(hc[b], kTcK);
    }
    U = hb[nblk];
    nks = hk[nblk];
    ucol = (int32_t*)dev_alloc(c, std::max<int64_t>(U, 1) * sizeof(int32_t));
    if (!ucol) return set_error(c, GM_E_NOMEM, "tensor-core tile union");
    if (!ensure(c, c->tc_kbase, (nblk + 1) * sizeof(int64_t)) ||
        !ensure(c, c->tc_upad, std::max<int64_t>(nks, 1) * kTcK * sizeof(int32_t)) ||
        !ensure(c, c->tc_img, std::max<int64_t>(nks, 1) * 3 * kTcA))
      return set_error(c, GM_E_NOMEM, "tensor-core tiles");
    GM_CUDA_CHECK(c, cudaMemcpyAsync(bptr, hb.data(), (nblk + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, st));
    GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_kbase.p, hk.data(), (nblk + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, st));
    GM_PROF(c, "k_tc_union");
    k_tc_union<<<(unsigned)nblk, 256, bm_smem, st>>>(
        n, 1, c->row_ptr, c->col, (const int64_t*)c->tc_brow0.p, trow, nullptr, bptr,
        (const int64_t*)c->tc_kbase.p, ucol, (int32_t*)c->tc_upad.p);
    GM_LAUNCH_CHECK(c);
  } else {
    int64_t n_pad = 1024;
    while (n_pad < nnz) n_pad <<= 1;
    ScopedDev kd(c, n_pad * sizeof(unsigned long long));
    ScopedDev fd(c, std::max<int64_t>(nnz, 1) * sizeof(int64_t));
    ScopedDev pd(c, (nnz + 1) * sizeof(int64_t));
    if (!kd.p || !fd.p || !pd.p) return set_error(c, GM_E_NOMEM, "tensor-core tile keys");
    unsigned long long* keys = (unsigned long long*)kd.p;
    int64_t* flag = (int64_t*)fd.p;
    int64_t* pos = (int64_t*)pd.p;
    GM_PROF(c, "k_tc_keys");
    k_tc_keys<<<wb, 256, 0, st>>>(n, c->row_ptr, c->col, nnz, n_pad, tb, tpos, keys);
    GM_LAUNCH_CHECK(c);
    gm_status s = sort_u64(c, keys, n_pad);
    if (s != GM_OK) return s;
    GM_PROF(c, "k_tc_flags");
    k_tc_flags<<<eb, 256, 0, st>>>(nnz, keys, flag);
    GM_LAUNCH_CHECK(c);
    s = scan_i64(c, flag, pos, nnz);
    if (s != GM_OK) return s;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(&U, pos + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
    ucol = (int32_t*)dev_alloc(c, std::max<int64_t>(U, 1) * sizeof(int32_t));
    ScopedDev ub(c, std::max<int64_t>(U, 1) * sizeof(int32_t));
    if (!ucol || !ub.p) return set_error(c, GM_E_NOMEM, "tensor-core tile union");
    int32_t* ublk = (int32_t*)ub.p;
    GM_PROF(c, "k_tc_unique");
    k_tc_unique<<<eb, 256, 0, st>>>(nnz, keys, flag, pos, ucol, ublk);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_tc_bptr");
    k_tc_bptr<<<(int)std::min<int64_t>(ceil_div(U + 1, 256), 16 * sms), 256, 0, st>>>(U, nblk,
                                                                                     ublk, bptr);
    GM_LAUNCH_CHECK(c);
    GM_CUDA_CHECK(c, cudaMemcpyAsync(hb.data(), bptr, (nblk + 1) * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
    for (int64_t b = 0; b < nblk; ++b) hk[b + 1] = hk[b] + ceil_div(hb[b + 1] - hb[b], kTcK);
    nks = hk[nblk];
    if (!ensure(c, c->tc_kbase, (nblk + 1) * sizeof(int64_t)) ||
        !ensure(c, c->tc_upad, std::max<int64_t>(nks, 1) * kTcK * sizeof(int32_t)) ||
        !ensure(c, c->tc_img, std::max<int64_t>(nks, 1) * 3 * kTcA))
      return set_error(c, GM_E_NOMEM, "tensor-core tiles");
    GM_CUDA_CHECK(c, cudaMemcpyAsync(c->tc_kbase.p, hk.data(), (nblk + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, st));
    GM_PROF(c, "k_tc_ucol");
    k_tc_ucol<<<(int)std::min<int64_t>(nblk, 16 * sms), 256, 0, st>>>(
        nblk, bptr, (const int64_t*)c->tc_kbase.p, ucol, (int32_t*)c->tc_upad.p);
    GM_LAUNCH_CHECK(c);
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));  // the scoped scratch is released here
  }
  int64_t* kbase = (int64_t*)c->tc_kbase.p;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->tc_img.p, 0, (size_t)nks * 3 * kTcA, st));
  GM_PROF(c, "k_tc_fill");
  k_tc_fill<<<wb, 256, 0, st>>>(n, c->row_ptr, c->col, (const float*)c->val, bptr, kbase, ucol,
                                tb, tpos, (const int64_t*)c->tc_brow0.p,
                                (unsigned char*)c->tc_img.p);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  dev_free_now(c, bptr, (nblk + 1) * sizeof(int64_t));
  dev_free_now(c, ucol, std::max<int64_t>(U, 1) * sizeof(int32_t));
  c->tc_nblk = nblk;
  c->tc_nks = nks;
  c->stats.tile_ksteps = nks;
  return GM_OK;
}

static gm_status launch_tc(gm_ctx* c, int pf, dim3 grid, int64_t n, int R, const float* dv,
                           const float* P, const float* PD, float* Q, double* part_pq,
                           TcPanels pk, int64_t pd_elems, cudaStream_t st,
                           bool planes_ready = false) {
  const int64_t* kb = (const int64_t*)c->tc_kbase.p;
  const int32_t* up = (const int32_t*)c->tc_upad.p;
  const uint4* im = (const uint4*)c->tc_img.p;
  if (pf == 4) {
    // BF16 planes of PD, then the product with B copied straight from them
    if (!ensure(c, c->tc_planes, (size_t)std::max<int64_t>(pd_elems, 1) * 3 * sizeof(uint16_t)))
      return set_error(c, GM_E_NOMEM, "BF16 planes of the panel");
    uint16_t* pl = (uint16_t*)c->tc_planes.p;
    const int sb = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(pd_elems, 4 * 256), 1),
                                          8 * sm_count(c));
    // per-kernel timing only for the single-panel path (the packed path may
    // run inside a graph capture)
    if (!planes_ready) {
      if (!pk.items) GM_PROF(c, "k_split3_planes");
      k_split3_planes<<<sb, 256, 0, st>>>(pd_elems, PD, pl);
    }
    if (!pk.items) GM_PROF(c, "k_panel_spmm_tc");
    const unsigned char* ib = (const unsigned char*)c->tc_img.p;
    if (c->cfg.tc_products == 3)
      k_panel_spmm_tc_async<3><<<grid, kTaThreads, kTaSmem, st>>>(
          n, R, kb, up, ib, dv, P, pl, pd_elems, Q, part_pq, pk, c->d_flags);
    else
      k_panel_spmm_tc_async<6><<<grid, kTaThreads, kTaSmem, st>>>(
          n, R, kb, up, ib, dv, P, pl, pd_elems, Q, part_pq, pk, c->d_flags);
    return GM_OK;
  }
  if (c->cfg.tc_products == 3) {
    if (pf == 3)
      k_panel_spmm_tc_ws<3><<<grid, 288, kTcSmemWs, st>>>(n, R, kb, up, im, dv, P, PD, Q,
                                                          part_pq, pk, c->d_flags);
    else if (pf == 2)
      k_panel_spmm_tc<2, 3><<<grid, 256, kTcSmem, st>>>(n, R, kb, up, im, dv, P, PD, Q, part_pq,
                                                        pk, c->d_flags);
    else
      k_panel_spmm_tc<1, 3><<<grid, 256, kTcSmem, st>>>(n, R, kb, up, im, dv, P, PD, Q, part_pq,
                                                        pk, c->d_flags);
    return GM_OK;
  }
  if (pf == 3)
    k_panel_spmm_tc_ws<6><<<grid, 288, kTcSmemWs, st>>>(n, R, kb, up, im, dv, P, PD, Q, part_pq,
                                                        pk, c->d_flags);
  else if (pf == 2)
    k_panel_spmm_tc<2, 6><<<grid, 256, kTcSmem, st>>>(n, R, kb, up, im, dv, P, PD, Q, part_pq, pk,
                                                      c->d_flags);
  else
    k_panel_spmm_tc<1, 6><<<grid, 256, kTcSmem, st>>>(n, R, kb, up, im, dv, P, PD, Q, part_pq, pk,
                                                      c->d_flags);
  return GM_OK;
}

// Variant of the tile product: 1, 2 = CTA-synchronous with gathers one or two
// steps ahead, 3 = warp-specialised ring, 4 = B copied asynchronously from
// BF16 planes of PD.  GM_TC_PREFETCH=1|2|3|4 pins it, else the fastest on the
// context's first panel product of the width class whose slot `variant` is
// (two timed launches each; the product is idempotent: Q is overwritten).
static gm_status tc_tune(gm_ctx* c, dim3 grid, int64_t n, int R, const float* dv, const float* P,
                         const float* PD, float* Q, double* part_pq, TcPanels pk,
                         int64_t pd_elems, int& variant) {
  if (variant) return GM_OK;
  // the planes are allocated here, before any graph capture of the products
  if (!ensure(c, c->tc_planes, (size_t)std::max<int64_t>(pd_elems, 1) * 3 * sizeof(uint16_t)))
    return set_error(c, GM_E_NOMEM, "BF16 planes of the panel");
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc_async<6>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTaSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc_async<3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTaSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc<1, 6>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc<2, 6>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc_ws<6>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemWs));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc<1, 3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc<2, 3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  GM_CUDA_CHECK(c, cudaFuncSetAttribute(k_panel_spmm_tc_ws<3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemWs));
  if (const char* e = std::getenv("GM_TC_PREFETCH")) {
    const int v = std::atoi(e);
    if (v >= 1 && v <= 4) {
      variant = v;
      return GM_OK;
    }
  }
  cudaEvent_t a, b;
  GM_CUDA_CHECK(c, cudaEventCreate(&a));
  GM_CUDA_CHECK(c, cudaEventCreate(&b));
  float best = 1e30f;
  // two timed launches per variant, the faster kept: a single launch is
  // cold (instruction cache, first touch of the planes) and misranks them
  for (int pf : {1, 2, 3, 4}) {
    float fastest = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      float ms = 0;
      GM_CUDA_CHECK(c, cudaEventRecord(a, c->stream));
      gm_status ls = launch_tc(c, pf, grid, n, R, dv, P, PD, Q, part_pq, pk, pd_elems, c->stream);
      if (ls != GM_OK) return ls;
      GM_CUDA_CHECK(c, cudaEventRecord(b, c->stream));
      GM_CUDA_CHECK(c, cudaEventSynchronize(b));
      GM_LAUNCH_CHECK(c);
      GM_CUDA_CHECK(c, cudaEventElapsedTime(&ms, a, b));
      fastest = std::min(fastest, ms);
    }
    if (fastest < best) {
      best = fastest;
      variant = pf;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return GM_OK;
}

gm_status panel_spmm_tc(gm_ctx* c, int64_t n, int R, const float* dv, const float* P,
                        const float* PD, float* Q, double* part_pq, bool planes_ready) {
  // column groups vary fastest: the CTAs resident together share their row
  // blocks' tile images (read from DRAM once instead of once per group)
  dim3 grid((unsigned)ceil_div(R, kTcCols), (unsigned)c->tc_nblk);
  const TcPanels pk{nullptr, nullptr, nullptr, nullptr,
                    c->tc_order ? (const int32_t*)c->tc_trow.p : nullptr};
  // one column group (the deflation refresh's 64-column products) and wider
  // panels are tuned apart: their grids differ by the number of groups
  int& variant = R <= kTcCols ? c->tc_pf_narrow : c->tc_pf;
  gm_status s = tc_tune(c, grid, n, R, dv, P, PD, Q, part_pq, pk, n * (int64_t)R, variant);
  if (s != GM_OK) return s;
  if (variant != 4) GM_PROF(c, "k_panel_spmm_tc");  // variant 4 times its two kernels itself
  s = launch_tc(c, variant, grid, n, R, dv, P, PD, Q, part_pq, pk, n * (int64_t)R, c->stream,
                planes_ready && variant == 4);
  if (s != GM_OK) return s;
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

int tc_variant(gm_ctx* c, int R) { return R <= kTcCols ? c->tc_pf_narrow : c->tc_pf; }

// Packed multi-field panels: one CTA per (tile block, column group) item.
gm_status panel_spmm_tc_packed(gm_ctx* c, int64_t n_items, const int2* items,
                               const int64_t* blk_base, const int32_t* blk_width, const float* dv,
                               const float* P, const float* PD, float* Q, int64_t pd_elems,
                               cudaStream_t st, bool tune) {
  const TcPanels pk{blk_base, blk_width, (const int64_t*)c->tc_brow0.p, items,
                    c->tc_order ? (const int32_t*)c->tc_trow.p : nullptr};
  dim3 grid((unsigned)n_items);
  if (tune) return tc_tune(c, grid, c->n, 0, dv, P, PD, Q, nullptr, pk, pd_elems, c->tc_pf);
  return launch_tc(c, c->tc_pf, grid, c->n, 0, dv, P, PD, Q, nullptr, pk, pd_elems, st);
}

}  // namespace gm
