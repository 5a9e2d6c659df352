// Learned surrogate of the pair covariance: a 5-64-64-64-2 SiLU MLP on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulators in
// tensor memory).  It maps the scale-free geometry of a pair of sightlines
// and the hyperparameters to y = ln K (K = log1p(R) before the taper) and to
// e, an estimate of ln |y_pred - y|.  Pairs whose estimated error exceeds the
// gate fall back to the sightline quadrature.  The paper computes every
// entry by the sightline integral (Sect. 3); the surrogate approximates it.
//
// Inference tile: 128 pairs (one per thread of a 4-warp block), M = 128.
//   layer 1: [128 x 16] x [16 x 64]   (5 features padded to K = 16)
//   layers 2, 3: [128 x 64] x [64 x 64]  (four K = 16 steps)
//   layer 4: [128 x 64] x [64 x 16]   (2 outputs padded to N = 16)
// Operands live in shared memory in the no-swizzle K-major layout of 8 x 16 B
// core matrices; one thread issues tcgen05.mma, tcgen05.commit signals an
// mbarrier, and the four warps read the accumulator rows with tcgen05.ld,
// add the bias, apply SiLU and write the next layer's operand.
//
// Precision: every operand (features, activations, weights) is held as two
// BF16 pieces x = x_hi + x_lo (x_hi = x rounded to BF16, x_lo = the rounded
// remainder) and each product is x_hi y_hi + x_hi y_lo + x_lo y_hi (three
// MMAs, FP32 accumulation): about 2^-16 relative, so the network's output is
// that of its FP32 weights to ~1e-4 in ln K.  A single BF16 piece (2^-8 per
// operand) limited the served entries to ~1 % in K, the scale of the
// network's own fit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kMlpIn = 5, kMlpHid = 64, kMlpOut = 2;
// parameter vector layout (FP32): W1 [5][64], b1[64], W2 [64][64], b2, W3, b3,
// W4 [64][2], b4[2]  (W[k][n]: input k -> output n)
constexpr int kW1 = 0, kB1 = kW1 + kMlpIn * kMlpHid, kW2 = kB1 + kMlpHid,
              kB2 = kW2 + kMlpHid * kMlpHid, kW3 = kB2 + kMlpHid,
              kB3 = kW3 + kMlpHid * kMlpHid, kW4 = kB3 + kMlpHid,
              kB4 = kW4 + kMlpHid * kMlpOut, kMlpParams = kB4 + kMlpOut;

// Shared-memory operand images (bytes).
constexpr int kSW1 = 64 * 16 * 2;    // B of layer 1: 64 rows (n) x 16 (k)
constexpr int kSW = 64 * 64 * 2;     // B of layers 2, 3
constexpr int kSW4 = 16 * 64 * 2;    // B of layer 4: 16 rows x 64
constexpr int kSA1 = 128 * 16 * 2;   // A of layer 1
constexpr int kSA = 128 * 64 * 2;    // A of layers 2-4
constexpr int kSWimg = kSW1 + 2 * kSW + kSW4;  // one piece of all weight images (20 KB)
// training: transposed weight images of the backward pass, and the dOut image
constexpr int kSWb4 = 64 * 16 * 2, kSWb = 64 * 64 * 2;
constexpr int kSWbimg = kSWb4 + 2 * kSWb;  // 18 KB per piece
constexpr int kSD = 128 * 16 * 2;          // dOut image (128 samples x 16)

// byte offset of element (row, k) in a K-major no-swizzle image with K_total
// columns: core matrices of 8 rows x 8 elements (16 B rows), k-adjacent
// core matrices 128 B apart (LBO), 8-row groups K_total/8 * 128 B apart (SBO)
__host__ __device__ __forceinline__ int kmaj_off(int row, int k, int ktot) {
  return (row >> 3) * (ktot / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;                // base offset 0, swizzle none
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      mbar));
}

// Bounded wait on an mbarrier phase; returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase));
    if (done) return true;
  }
  return false;
}

// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

struct MlpIn {
  const double* si;      // per pair, or null with row/col arrays below
  const double* sj;
  const double* chord;
  int64_t n;
  double sigma2;
  double L0;
};

// Scale-free geometry of a pair in units of L0: ln(mean distance)/4, offset
// along the sightlines /3, transverse offset at the mean distance /3, then
// sigma2 and ln(L0 / 20 pc).
__device__ __forceinline__ void pair_features(double si, double sj, double chord, double sigma2,
                                              double L0, float* f) {
  const double g = sqrt(si * sj) / L0;
  f[0] = (float)(0.25 * log(g));
  f[1] = (float)(fabs(si - sj) / (3.0 * L0));
  f[2] = (float)(chord * g / 3.0);
  f[3] = (float)sigma2;
  f[4] = (float)log(L0 / 20.0);
}

// Two BF16 pieces of x, packed in pairs: hi = x rounded to BF16 (nearest
// even), lo = the remainder x - hi rounded the same way.
__device__ __forceinline__ void split2_pack(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Writes 8 consecutive values of one row (k = 8 g ..) of a K-major operand,
// both pieces (the lo image `lo_off` bytes after the hi image).
__device__ __forceinline__ void store8_split(unsigned char* img, int lo_off, int off, const float* v) {
  uint4 uh, ul;
  split2_pack(v[0], v[1], uh.x, ul.x);
  split2_pack(v[2], v[3], uh.y, ul.y);
  split2_pack(v[4], v[5], uh.z, ul.z);
  split2_pack(v[6], v[7], uh.w, ul.w);
  *reinterpret_cast<uint4*>(img + off) = uh;
  *reinterpret_cast<uint4*>(img + lo_off + off) = ul;
}

// Writes one thread's 64 activations (row `row`) into a K = 64 operand image
// (hi piece at sA, lo piece at sA + kSA).
__device__ __forceinline__ void store_row64(unsigned char* sA, int row, const float* h) {
#pragma unroll
  for (int g = 0; g < 8; ++g) store8_split(sA, kSA, kmaj_off(row, 8 * g, 64), h + 8 * g);
}

// Forward pass over a list of pairs; writes y and e.  Block = 128 threads.
// Weights: operand images (BF16) prepared by k_mlp_pack, biases FP32.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpIn in, const unsigned char* __restrict__ wimg,
                                                     const float* __restrict__ params,
                                                     float* __restrict__ y_out,
                                                     float* __restrict__ e_out,
                                                     unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // weight images: hi pieces (20 KB) then lo pieces (20 KB)
  unsigned char* sW1 = smem;                 // 2 KB
  unsigned char* sW2 = sW1 + kSW1;           // 8 KB
  unsigned char* sW3 = sW2 + kSW;            // 8 KB
  unsigned char* sW4 = sW3 + kSW;            // 2 KB
  unsigned char* sA1 = smem + 2 * kSWimg;    // 4 KB hi + 4 KB lo
  unsigned char* sA = sA1 + 2 * kSA1;        // 16 KB hi + 16 KB lo
  float* sBias = reinterpret_cast<float*>(sA + 2 * kSA);  // 64*3 + 2
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5;
  // weights and biases into shared memory
  for (int k = tid; k < 2 * kSWimg / 16; k += blockDim.x)
    reinterpret_cast<uint4*>(smem)[k] = reinterpret_cast<const uint4*>(wimg)[k];
  for (int k = tid; k < kMlpHid; k += blockDim.x) {
    sBias[k] = params[kB1 + k];
    sBias[64 + k] = params[kB2 + k];
    sBias[128 + k] = params[kB3 + k];
  }
  if (tid < kMlpOut) sBias[192 + tid] = params[kB4 + tid];
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes
  const uint32_t mb = smem_u32(&mbar);
  uint32_t phase = 0;

  const uint32_t dA1 = smem_u32(sA1), dA = smem_u32(sA);
  const uint32_t dW1 = smem_u32(sW1), dW2 = smem_u32(sW2), dW3 = smem_u32(sW3),
                 dW4 = smem_u32(sW4);
  const uint32_t id64 = idesc_bf16(128, 64), id16 = idesc_bf16(128, 16);

  const int64_t ntiles = (in.n + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * 128 + tid;
    // layer-1 operand: 5 features, zero padded to 16
    {
      float f[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) f[k] = 0.f;
      if (p < in.n) pair_features(in.si[p], in.sj[p], in.chord[p], in.sigma2, in.L0, f);
#pragma unroll
      for (int g = 0; g < 2; ++g) store8_split(sA1, kSA1, kmaj_off(tid, 8 * g, 16), f + 8 * g);
    }
    for (int layer = 0; layer < 4; ++layer) {
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        // per K-step: the two small cross terms, then hi x hi
        if (layer == 0) {
          mma_bf16(tmem, mdesc(dA1 + kSA1, 128, 256), mdesc(dW1, 128, 256), id64, 0);
          mma_bf16(tmem, mdesc(dA1, 128, 256), mdesc(dW1 + kSWimg, 128, 256), id64, 1);
          mma_bf16(tmem, mdesc(dA1, 128, 256), mdesc(dW1, 128, 256), id64, 1);
        } else {
          const uint32_t dw = layer == 1 ? dW2 : (layer == 2 ? dW3 : dW4);
          const uint32_t idd = layer == 3 ? id16 : id64;
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const uint64_t ah = mdesc(dA + 256 * s, 128, 1024),
                           al = mdesc(dA + kSA + 256 * s, 128, 1024),
                           wh = mdesc(dw + 256 * s, 128, 1024),
                           wl = mdesc(dw + kSWimg + 256 * s, 128, 1024);
            mma_bf16(tmem, al, wh, idd, s > 0 ? 1u : 0u);
            mma_bf16(tmem, ah, wl, idd, 1u);
            mma_bf16(tmem, ah, wh, idd, 1u);
          }
        }
        mma_commit(mb);
      }
      const bool ok = mbar_wait(mb, phase);
      phase ^= 1;
      if (!ok) abort_flag = 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      if (abort_flag) break;
      if (layer < 3) {
        float h[64];
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_ld16(tmem_row + 16 * q, h + 16 * q);
        const float* bias = sBias + 64 * layer;
#pragma unroll
        for (int k = 0; k < 64; ++k) h[k] = silu_f(h[k] + bias[k]);
        store_row64(sA, tid, h);
      } else {
        float o[16];
        tmem_ld16(tmem_row, o);
        if (p < in.n) {
          y_out[p] = o[0] + sBias[192];
          e_out[p] = o[1] + sBias[193];
        }
      }
    }
    if (abort_flag) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(flags, kFlagTimeout);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
  }
}

// BF16 operand images of the weights (B operands are W^T, K-major), two
// pieces (hi image, then lo image kSWimg bytes later):
//   layer 1: rows n < 64, k < 16 (k >= 5 zero); layers 2, 3: 64 x 64;
//   layer 4: rows n < 16 (n >= 2 zero), k < 64.
__device__ __forceinline__ void put_split(unsigned char* img, int off, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(img + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(img + kSWimg + off) = __float2bfloat16_rn(v - __bfloat162float(h));
}

__global__ void k_mlp_pack(const float* __restrict__ params, unsigned char* __restrict__ img) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < 64 * 64; idx += blockDim.x * gridDim.x) {
    const int n = idx / 64, k = idx % 64;
    if (k < 16) put_split(img, kmaj_off(n, k, 16), k < kMlpIn ? params[kW1 + k * kMlpHid + n] : 0.f);
    put_split(img, kSW1 + kmaj_off(n, k, 64), params[kW2 + k * kMlpHid + n]);
    put_split(img, kSW1 + kSW + kmaj_off(n, k, 64), params[kW3 + k * kMlpHid + n]);
    if (n < 16)
      put_split(img, kSW1 + 2 * kSW + kmaj_off(n, k, 64),
                n < kMlpOut ? params[kW4 + k * kMlpOut + n] : 0.f);
  }
}

constexpr size_t kMlpSmem = 2 * kSWimg + 2 * kSA1 + 2 * kSA + 256 * sizeof(float);

gm_status mlp_forward(gm_ctx* c, const MlpIn& in, float* y, float* e) {
  if (!c->mlp_params || !c->mlp_trained) return set_error(c, GM_E_STATE, "surrogate has no weights");
  if (in.n == 0) return GM_OK;
  GM_PROF(c, "k_mlp_pack");
  k_mlp_pack<<<16, 256, 0, c->stream>>>(c->mlp_params, c->mlp_img);
  GM_LAUNCH_CHECK(c);
  cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  const int64_t ntiles = (in.n + 127) / 128;
  const int blocks = (int)std::min<int64_t>(ntiles, 4 * sm_count(c));
  GM_PROF(c, "k_mlp_forward");
  k_mlp_forward<<<blocks, 128, kMlpSmem, c->stream>>>(in, c->mlp_img, c->mlp_params, y, e,
                                                     c->d_flags);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm

namespace gm {
static bool mlp_is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gm_status mlp_ensure(gm_ctx* c) {
  if (c->mlp_params) return GM_OK;
  c->mlp_params = (float*)dev_alloc(c, kMlpParams * sizeof(float));
  c->mlp_img = (unsigned char*)dev_alloc(c, 2 * kSWimg);
  c->mlp_bimg = (unsigned char*)dev_alloc(c, 2 * kSWbimg);
  if (!c->mlp_params || !c->mlp_img || !c->mlp_bimg)
    return set_error(c, GM_E_NOMEM, "surrogate weights");
  return GM_OK;
}
}  // namespace gm

using namespace gm;

extern "C" int64_t gm_surrogate_param_count(void) { return kMlpParams; }

extern "C" gm_status gm_surrogate_set_params(gm_ctx* c, const float* params, int64_t n) {
  if (!c || !params || n != kMlpParams) return GM_E_INVAL;
  gm_status st = mlp_ensure(c);
  if (st != GM_OK) return st;
  cudaMemcpyKind k = mlp_is_dev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->mlp_params, params, n * sizeof(float), k, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  c->mlp_trained = true;
  return GM_OK;
}

extern "C" gm_status gm_surrogate_get_params(gm_ctx* c, float* out, int64_t n) {
  if (!c || !out || n != kMlpParams) return GM_E_INVAL;
  if (!c->mlp_params || !c->mlp_trained) return set_error(c, GM_E_STATE, "surrogate has no weights");
  cudaMemcpyKind k = mlp_is_dev(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(out, c->mlp_params, n * sizeof(float), k, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

extern "C" gm_status gm_surrogate_eval(gm_ctx* c, int64_t n, const double* si, const double* sj,
                                       const double* chord, double sigma2, double L0,
                                       float* y_out, float* e_out) {
  if (!c || n < 0 || (n > 0 && (!si || !sj || !chord || !y_out || !e_out))) return GM_E_INVAL;
  if (!(sigma2 > 0) || !(L0 > 0)) return GM_E_INVAL;
  if (n == 0) return GM_OK;
  c->launches = 0;
  const size_t nb = (size_t)n * sizeof(double);
  double* buf = (double*)dev_alloc(c, 3 * nb + 2 * (size_t)n * sizeof(float));
  if (!buf) return set_error(c, GM_E_NOMEM, "surrogate eval staging");
  const double* src[3] = {si, sj, chord};
  for (int k = 0; k < 3; ++k) {
    cudaMemcpyKind kind = mlp_is_dev(src[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(buf + k * n, src[k], nb, kind, c->stream));
  }
  float* y = (float*)(buf + 3 * n);
  float* e = y + n;
  MlpIn in{buf, buf + n, buf + 2 * n, n, sigma2, L0};
  gm_status st = mlp_forward(c, in, y, e);
  if (st != GM_OK) return st;
  cudaMemcpyKind ky = mlp_is_dev(y_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaMemcpyKind ke = mlp_is_dev(e_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(y_out, y, n * sizeof(float), ky, c->stream));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(e_out, e, n * sizeof(float), ke, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, buf, 3 * nb + 2 * (size_t)n * sizeof(float));
  unsigned* h = (unsigned*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  if (*h & kFlagTimeout) {
    cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream);
    return set_error(c, GM_E_TIMEOUT, "tensor-core pipeline wait expired");
  }
  return GM_OK;
}

// ---------------------------------------------------------------------------
// Training (FP32 on the CUDA cores): targets from the sightline quadrature,
// loss  mean (y - ln K)^2 + lambda mean rho_q(ln(|y - ln K| + 1e-5) - e), with
// rho_q(u) = u (q - [u < 0]) the pinball loss at q = 0.95 (so that e tracks an
// upper quantile of the log error, not its mean) and the error target held
// fixed; mini-batches drawn with replacement, Adam.
// ---------------------------------------------------------------------------
namespace gm {

constexpr float kErrQuantile = 0.95f;

// SplitMix64 (Steele, Lea & Flood 2014): a counter-based stream of 64-bit words.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double u01(uint64_t seed, uint64_t i, uint64_t k) {
  return (double)(splitmix64(seed ^ splitmix64(i * 8 + k)) >> 11) * (1.0 / 9007199254740992.0);
}

// Training pairs like those of the covariance: s_i log-uniform in
// [s_min, s_max]; s_j = s_i + delta, delta uniform in [-c, c] (clipped at
// s_min / 2); squared 3-D separation uniform in [delta^2, c^2].
__global__ void k_mlp_sample(int64_t n, uint64_t seed, double s_min, double s_max, double cut,
                             double* __restrict__ si, double* __restrict__ sj,
                             double* __restrict__ chord) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double a = exp(log(s_min) + (log(s_max) - log(s_min)) * u01(seed, p, 0));
    double b = a + cut * (2.0 * u01(seed, p, 1) - 1.0);
    b = fmax(b, 0.5 * s_min);
    const double dl = b - a;
    const double d2 = dl * dl + (cut * cut - dl * dl) * u01(seed, p, 2);
    si[p] = a;
    sj[p] = b;
    chord[p] = sqrt(fmax(d2 - dl * dl, 0.0) / (a * b));
  }
}

// Training pairs drawn from the catalogue's own neighbour pairs: the CSR of
// nq query stars (their s, u in qs, qux, ...) against all stars; pair p is
// entry e = uniform in [0, qnnz) (self pairs, at zero separation, are always
// computed by the quadrature and are redrawn).
__global__ void k_mlp_sample_cat(int64_t n, uint64_t seed, int64_t nq, int64_t qnnz,
                                 const int64_t* __restrict__ qptr, const int32_t* __restrict__ qcol,
                                 const double* __restrict__ qs, const double* __restrict__ qux,
                                 const double* __restrict__ quy, const double* __restrict__ quz,
                                 const double* __restrict__ s, const double* __restrict__ ux,
                                 const double* __restrict__ uy, const double* __restrict__ uz,
                                 double* __restrict__ si, double* __restrict__ sj,
                                 double* __restrict__ chord) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double a = 0, b = 0, ch = 0;
    for (int tries = 0; tries < 8; ++tries) {
      const int64_t e = (int64_t)(splitmix64(seed ^ splitmix64(p * 16 + tries)) % (uint64_t)qnnz);
      int64_t lo = 0, hi = nq;  // row of entry e
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (qptr[mid] <= e) lo = mid; else hi = mid;
      }
      const int32_t j = qcol[e];
      const double dx = qux[lo] - ux[j], dy = quy[lo] - uy[j], dz = quz[lo] - uz[j];
      a = qs[lo];
      b = s[j];
      ch = sqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
      if (ch > 0.0 || a != b) break;
    }
    si[p] = a;
    sj[p] = b;
    chord[p] = ch;
  }
}

__global__ void k_gather_rows(int64_t nq, int64_t n, const double* __restrict__ s,
                              const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ uz, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nq;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (k * n) / nq;  // evenly spread over the spatially sorted stars
    out[k] = s[i];
    out[nq + k] = ux[i];
    out[2 * nq + k] = uy[i];
    out[3 * nq + k] = uz[i];
  }
}

__global__ void k_mlp_features(int64_t n, const double* __restrict__ si,
                               const double* __restrict__ sj, const double* __restrict__ chord,
                               const double* __restrict__ K, double sigma2, double L0,
                               float* __restrict__ X, float* __restrict__ Y) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float f[5];
    pair_features(si[p], sj[p], chord[p], sigma2, L0, f);
    for (int k = 0; k < 5; ++k) X[p * 5 + k] = f[k];
    Y[p] = (float)log(K[p]);
  }
}

__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float silu_exact(float z) { return z / (1.0f + expf(-z)); }

// Per batch sample (one thread): forward, loss terms, backward to dZ.
// Saves per sample: h0 (5), h1, h2, h3 (64 each), dz1, dz2, dz3 (64 each),
// dout (2) -> stride 5 + 6*64 + 2 = 391 floats.
constexpr int kSv = 5 + 6 * 64 + 2;
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(int64_t n_data, int B, int direct,
                                                     uint64_t seed, uint64_t step,
                                                     const float* __restrict__ X,
                                                     const float* __restrict__ Y,
                                                     const float* __restrict__ params, float lam,
                                                     float* __restrict__ save,
                                                     double* __restrict__ loss_part) {
  extern __shared__ float sp[];  // parameters
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) sp[k] = params[k];
  __syncthreads();
  const float* W1 = sp + kW1;
  const float* b1 = sp + kB1;
  const float* W2 = sp + kW2;
  const float* b2 = sp + kB2;
  const float* W3 = sp + kW3;
  const float* b3 = sp + kB3;
  const float* W4 = sp + kW4;
  const float* b4 = sp + kB4;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double l1 = 0, l2 = 0;
  if (s < B) {
    // sample s of the batch: data row s (direct) or a row drawn with replacement
    const int64_t p = direct ? (int64_t)s
                             : (int64_t)(splitmix64(seed ^ splitmix64(step * 1000003ull + s)) %
                                         (uint64_t)n_data);
    float* sv = save + (int64_t)s * kSv;
    float* h0 = sv;
    float* h1 = sv + 5;
    float* h2 = h1 + 64;
    float* h3 = h2 + 64;
    float* dz1 = h3 + 64;
    float* dz2 = dz1 + 64;
    float* dz3 = dz2 + 64;
    float* dout = dz3 + 64;
    float x[5];
    for (int k = 0; k < 5; ++k) h0[k] = x[k] = X[p * 5 + k];
    float z1[64], z2[64], z3[64];
    for (int nn = 0; nn < 64; ++nn) {
      float a = b1[nn];
      for (int k = 0; k < 5; ++k) a = fmaf(x[k], W1[k * 64 + nn], a);
      z1[nn] = a;
      h1[nn] = silu_exact(a);
    }
    for (int nn = 0; nn < 64; ++nn) {
      float a = b2[nn];
      for (int k = 0; k < 64; ++k) a = fmaf(h1[k], W2[k * 64 + nn], a);
      z2[nn] = a;
    }
    for (int nn = 0; nn < 64; ++nn) h2[nn] = silu_exact(z2[nn]);
    for (int nn = 0; nn < 64; ++nn) {
      float a = b3[nn];
      for (int k = 0; k < 64; ++k) a = fmaf(h2[k], W3[k * 64 + nn], a);
      z3[nn] = a;
    }
    for (int nn = 0; nn < 64; ++nn) h3[nn] = silu_exact(z3[nn]);
    float out[2];
    for (int o = 0; o < 2; ++o) {
      float a = b4[o];
      for (int k = 0; k < 64; ++k) a = fmaf(h3[k], W4[k * 2 + o], a);
      out[o] = a;
    }
    const float r = out[0] - Y[p];
    const float et = logf(fabsf(r) + 1e-5f);
    // pinball loss of the error head at quantile kErrQuantile: u > 0 when the
    // head under-estimates the error
    const float u = et - out[1];
    const float wq = u > 0.f ? kErrQuantile : kErrQuantile - 1.f;
    l1 = (double)r * r;
    l2 = (double)(u * wq);
    const float g0 = 2.0f * r / (float)B, g1 = -lam * wq / (float)B;
    dout[0] = g0;
    dout[1] = g1;
    for (int k = 0; k < 64; ++k) dz3[k] = (W4[k * 2] * g0 + W4[k * 2 + 1] * g1) * dsilu_f(z3[k]);
    for (int k = 0; k < 64; ++k) {
      float a = 0;
      for (int nn = 0; nn < 64; ++nn) a = fmaf(W3[k * 64 + nn], dz3[nn], a);
      dz2[k] = a * dsilu_f(z2[k]);
    }
    for (int k = 0; k < 64; ++k) {
      float a = 0;
      for (int nn = 0; nn < 64; ++nn) a = fmaf(W2[k * 64 + nn], dz2[nn], a);
      dz1[k] = a * dsilu_f(z1[k]);
    }
  }
  // block sums of the loss terms (fixed order)
  __shared__ double sh[2][4];
  for (int off = 16; off > 0; off >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    l2 += __shfl_xor_sync(0xffffffffu, l2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = l1;
    sh[1][threadIdx.x >> 5] = l2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    loss_part[2 * blockIdx.x] = sh[0][0] + sh[0][1] + sh[0][2] + sh[0][3];
    loss_part[2 * blockIdx.x + 1] = sh[1][0] + sh[1][1] + sh[1][2] + sh[1][3];
  }
}

// Weight gradients: block = one input row k of one layer; thread = output n.
// dW[k][n] = sum_s h_{l-1}[s][k] dz_l[s][n] (fixed order over s); bias rows
// (k = -1) sum dz_l.  Grid: 5 + 64 + 64 + 64 weight rows + 4 bias rows.
__global__ void k_mlp_wgrad(int B, const float* __restrict__ save, float* __restrict__ grad) {
  const int r = blockIdx.x, nn = threadIdx.x;
  int layer, k;  // row r -> (layer, input index or -1 for bias)
  if (r < 5) { layer = 0; k = r; }
  else if (r < 69) { layer = 1; k = r - 5; }
  else if (r < 133) { layer = 2; k = r - 69; }
  else if (r < 197) { layer = 3; k = r - 133; }
  else { layer = r - 197; k = -1; }
  const int nout = layer == 3 ? 2 : 64;
  if (nn >= nout) return;
  const int hoff = layer == 0 ? 0 : 5 + 64 * (layer - 1);        // input activations
  const int goff = layer == 3 ? 5 + 6 * 64 : 5 + 3 * 64 + 64 * layer;  // dz of this layer
  float acc = 0.f;
  for (int s = 0; s < B; ++s) {
    const float* sv = save + (int64_t)s * kSv;
    const float h = k < 0 ? 1.0f : sv[hoff + k];
    acc = fmaf(h, sv[goff + nn], acc);
  }
  const int wbase = layer == 0 ? kW1 : layer == 1 ? kW2 : layer == 2 ? kW3 : kW4;
  const int bbase = layer == 0 ? kB1 : layer == 1 ? kB2 : layer == 2 ? kB3 : kB4;
  if (k < 0) grad[bbase + nn] = acc;
  else grad[wbase + k * nout + nn] = acc;
}

// Adam (Kingma & Ba 2015) on all parameters.
__global__ void k_mlp_adam(int np, const float* __restrict__ g, float* __restrict__ p,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                           float b2, float c1, float c2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1 - b1) * gk;
    const float vk = b2 * v[k] + (1 - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
  }
}

}  // namespace gm

namespace gm {

__global__ void k_minmax_s(int64_t n, const double* __restrict__ s, double* __restrict__ out) {
  __shared__ double lo[256], hi[256];
  double a = INFINITY, b = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a = fmin(a, s[i]);
    b = fmax(b, s[i]);
  }
  lo[threadIdx.x] = a;
  hi[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + w]);
      hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = lo[0];
    out[1] = hi[0];
  }
}


// ---------------------------------------------------------------------------
// Training on the tensor cores: one CTA per batch tile of 128 samples.
// Forward as in k_mlp_forward (the pre-activations Z1..Z3 stay in tensor
// memory); backward dH_l = dZ_{l+1} W_{l+1}^T as M = 128 (samples) products
// with the transposed weight images of k_mlp_pack_bwd; weight gradients
// dW_l = H_{l-1}^T dZ_l as products over the 128 samples, reading the same
// activation images as MN-major operands (M = the layer's inputs, zero-
// padded rows of the M = 128 product are not read back); bias gradients are
// column sums of dZ_l (FP32 shuffle reduce-scatter, then per warp in smem).
// Every operand is held as two BF16 pieces (three MMAs per step, as in the
// forward).  The tile's gradient goes to its own partial row; a second kernel
// sums the rows in a fixed order.
// Backward weight images (B operands, K-major, two pieces each):
//   W4b: rows n = hidden (64), k = outputs (16, 2 used): element W4[n][k]
//   W3b, W2b: rows n = layer input (64), k = layer output (64): W[n][k]

__global__ void k_mlp_pack_bwd(const float* __restrict__ params, unsigned char* __restrict__ img) {
  for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < 64 * 64; idx += blockDim.x * gridDim.x) {
    const int n = idx / 64, k = idx % 64;
    auto put = [&](int off, float v) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      *reinterpret_cast<__nv_bfloat16*>(img + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(img + kSWbimg + off) =
          __float2bfloat16_rn(v - __bfloat162float(h));
    };
    if (k < 16) put(kmaj_off(n, k, 16), k < kMlpOut ? params[kW4 + n * kMlpOut + k] : 0.f);
    put(kSWb4 + kmaj_off(n, k, 64), params[kW3 + n * kMlpHid + k]);
    put(kSWb4 + kSWb + kmaj_off(n, k, 64), params[kW2 + n * kMlpHid + k]);
  }
}

// three-MMA product of two-piece operands: lo x hi, hi x lo, hi x hi
__device__ __forceinline__ void mma3(uint32_t d, uint64_t ah, uint64_t al, uint64_t bh,
                                     uint64_t bl, uint32_t idesc, uint32_t acc) {
  mma_bf16(d, al, bh, idesc, acc);
  mma_bf16(d, ah, bl, idesc, 1u);
  mma_bf16(d, ah, bh, idesc, 1u);
}

constexpr size_t kTrainSmem = 2 * kSWimg + 2 * kSWbimg + 2 * kSA1 + 3 * 2 * kSA + 2 * kSD +
                              (256 + 4 * 200) * sizeof(float);

__global__ void __launch_bounds__(128) k_mlp_train_tc(
    int64_t n_data, int B, int direct, uint64_t seed, uint64_t step, const float* __restrict__ X,
    const float* __restrict__ Y, const float* __restrict__ params,
    const unsigned char* __restrict__ wimg, const unsigned char* __restrict__ wbimg, float lam,
    float* __restrict__ grad_part, double* __restrict__ loss_part, unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sWf = smem;                         // forward weights, hi then lo
  unsigned char* sWb = sWf + 2 * kSWimg;             // backward weights, hi then lo
  unsigned char* sX = sWb + 2 * kSWbimg;             // X (hi, lo)
  unsigned char* sH1 = sX + 2 * kSA1;                // H1 then dZ1 (hi, lo)
  unsigned char* sH2 = sH1 + 2 * kSA;                // H2 then dZ2
  unsigned char* sH3 = sH2 + 2 * kSA;                // H3 then dZ3
  unsigned char* sD = sH3 + 2 * kSA;                 // dOut (hi, lo)
  float* sBias = reinterpret_cast<float*>(sD + 2 * kSD);  // 194
  float* sDb = sBias + 256;                          // [4 warps][194] bias-gradient partials
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ double sh_loss[2][4];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k = tid; k < 2 * kSWimg / 16; k += blockDim.x)
    reinterpret_cast<uint4*>(sWf)[k] = reinterpret_cast<const uint4*>(wimg)[k];
  for (int k = tid; k < 2 * kSWbimg / 16; k += blockDim.x)
    reinterpret_cast<uint4*>(sWb)[k] = reinterpret_cast<const uint4*>(wbimg)[k];
  for (int k = tid; k < kMlpHid; k += blockDim.x) {
    sBias[k] = params[kB1 + k];
    sBias[64 + k] = params[kB2 + k];
    sBias[128 + k] = params[kB3 + k];
  }
  if (tid < kMlpOut) sBias[192 + tid] = params[kB4 + tid];
  for (int k = tid; k < 4 * 200; k += blockDim.x) sDb[k] = 0.f;
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the sample of this thread (row tid of the tile)
  const int sidx = blockIdx.x * 128 + tid;
  const bool live = sidx < B;
  const int64_t p = !live ? 0
                  : direct ? (int64_t)sidx
                           : (int64_t)(splitmix64(seed ^ splitmix64(step * 1000003ull + sidx)) %
                                       (uint64_t)n_data);
  {
    float f[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] = 0.f;
    if (live)
      for (int k = 0; k < kMlpIn; ++k) f[k] = X[p * kMlpIn + k];
#pragma unroll
    for (int g = 0; g < 2; ++g) store8_split(sX, kSA1, kmaj_off(tid, 8 * g, 16), f + 8 * g);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  // tensor-memory columns: Z1, Z2, Z3 at 0, 64, 128 (64 * layer), then the rest
  constexpr uint32_t cZ1 = 0, cOut = 192, cDH = 208, cW1 = 272, cW2 = 336,
                     cW3 = 400, cW4 = 464;
  const uint32_t mb = smem_u32(&mbar);
  uint32_t phase = 0;
  // MMAs issued by thread 0, then all threads wait; smem written by the
  // threads before is published to the tensor core first
  auto run = [&](auto&& issue) -> bool {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      issue();
      mma_commit(mb);
    }
    const bool ok = mbar_wait(mb, phase);
    phase ^= 1;
    if (!ok) abort_flag = 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    return !abort_flag;
  };
  const uint32_t id64 = idesc_bf16(128, 64), id16 = idesc_bf16(128, 16);
  const uint32_t idT64 = id64 | (1u << 15) | (1u << 16), idT16 = id16 | (1u << 15) | (1u << 16);
  const uint32_t aX = smem_u32(sX), aH1 = smem_u32(sH1), aH2 = smem_u32(sH2), aH3 = smem_u32(sH3),
                 aD = smem_u32(sD), aWf = smem_u32(sWf), aWb = smem_u32(sWb);
  // K-major operand of K = 64 (activation rows or weights), K-step s
  auto km64 = [](uint32_t a, int s) { return mdesc(a + 256 * s, 128, 1024); };
  // the same activation image as an MN-major operand over the samples:
  // K-step s of 16 samples, 8-column chunks 128 B apart, 8-sample groups 1 KB apart
  auto mn64 = [](uint32_t a, int s) { return mdesc(a + 2048 * s, 1024, 128); };
  auto mn16 = [](uint32_t a, int s) { return mdesc(a + 512 * s, 256, 128); };
  bool ok = true;
  float z[64];
  // ---- forward
  ok = ok && run([&] {
    mma3(tmem + cZ1, mdesc(aX, 128, 256), mdesc(aX + kSA1, 128, 256), mdesc(aWf, 128, 256),
         mdesc(aWf + kSWimg, 128, 256), id64, 0u);
  });
  const uint32_t wf[3] = {aWf + kSW1, aWf + kSW1 + kSW, aWf + kSW1 + 2 * kSW};  // W2, W3, W4
  unsigned char* sH[3] = {sH1, sH2, sH3};
  const uint32_t aH[3] = {aH1, aH2, aH3};
  for (int layer = 0; layer < 3 && ok; ++layer) {
    // H_layer = silu(Z_layer + b) into its image, then Z_{layer+1}
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + 64 * layer + 16 * q, z + 16 * q);
#pragma unroll
    for (int k = 0; k < 64; ++k) z[k] = silu_f(z[k] + sBias[64 * layer + k]);
    store_row64(sH[layer], tid, z);
    const uint32_t dcol = layer < 2 ? 64 * (layer + 1) : cOut;
    const uint32_t idd = layer < 2 ? id64 : id16;
    const uint32_t aa = aH[layer], ww = wf[layer];
    ok = run([&] {
      for (int s = 0; s < 4; ++s)
        mma3(tmem + dcol, km64(aa, s), km64(aa + kSA, s), km64(ww, s), km64(ww + kSWimg, s), idd,
             s > 0 ? 1u : 0u);
    });
  }
  // ---- loss and dOut
  double l1 = 0, l2 = 0;
  if (ok) {
    float o[16];
    tmem_ld16(tmem + lane_off + cOut, o);
    float d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) d[k] = 0.f;
    if (live) {
      const float out0 = o[0] + sBias[192], out1 = o[1] + sBias[193];
      const float r = out0 - Y[p];
      const float et = logf(fabsf(r) + 1e-5f);
      const float u = et - out1;
      const float wq = u > 0.f ? kErrQuantile : kErrQuantile - 1.f;
      l1 = (double)r * r;
      l2 = (double)(u * wq);
      d[0] = 2.0f * r / (float)B;
      d[1] = -lam * wq / (float)B;
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) store8_split(sD, kSD, kmaj_off(tid, 8 * g, 16), d + 8 * g);
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // output bias gradients
      float v = d[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) sDb[warp * 200 + 192 + k] = v;
    }
  }
  // ---- backward: dH3 = dOut W4^T and dW4 = H3^T dOut
  ok = ok && run([&] {
    mma3(tmem + cDH, mdesc(aD, 128, 256), mdesc(aD + kSD, 128, 256), mdesc(aWb, 128, 256),
         mdesc(aWb + kSWbimg, 128, 256), id64, 0u);
    for (int s = 0; s < 8; ++s)
      mma3(tmem + cW4, mn64(aH3, s), mn64(aH3 + kSA, s), mn16(aD, s), mn16(aD + kSD, s), idT16,
           s > 0 ? 1u : 0u);
  });
  // dZ_l = dH_l o silu'(Z_l + b_l) over the activation image of H_l, then
  // dH_{l-1} = dZ_l W_l^T and dW_l = H_{l-1}^T dZ_l
  const uint32_t wb[2] = {aWb + kSWb4, aWb + kSWb4 + kSWb};  // W3b, W2b
  const uint32_t cW[3] = {cW1, cW2, cW3};
  for (int layer = 2; layer >= 0 && ok; --layer) {
    float dh[64];
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + cDH + 16 * q, dh + 16 * q);
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + 64 * layer + 16 * q, z + 16 * q);
#pragma unroll
    for (int k = 0; k < 64; ++k) dh[k] *= dsilu_f(z[k] + sBias[64 * layer + k]);
    store_row64(sH[layer], tid, dh);
    // bias gradients: column sums over the warp's rows (reduce-scatter of 16
    // columns at a time), accumulated per warp
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
      float v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = dh[16 * c16 + k];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bool up = lane & 16;
        const float send = up ? v[j] : v[j + 8];
        v[j] = (up ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool up = lane & 8;
        const float send = up ? v[j] : v[j + 4];
        v[j] = (up ? v[j + 4] : v[j]) + __shfl_xor_sync(0xffffffffu, send, 8);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool up = lane & 4;
        const float send = up ? v[j] : v[j + 2];
        v[j] = (up ? v[j + 2] : v[j]) + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        v[0] = (up ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
      }
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
      const int colw = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                       ((lane >> 1) & 1);
      if ((lane & 1) == 0) sDb[warp * 200 + 64 * layer + 16 * c16 + colw] = v[0];
    }
    const uint32_t az = aH[layer];  // now dZ_layer
    const uint32_t ain = layer > 0 ? aH[layer - 1] : aX;
    const uint32_t cw = cW[layer];
    const int lyr = layer;
    ok = run([&] {
      if (lyr > 0) {  // dH_{layer-1} = dZ_layer W_layer^T
        const uint32_t bw = wb[2 - lyr];
        for (int s = 0; s < 4; ++s)
          mma3(tmem + cDH, km64(az, s), km64(az + kSA, s), km64(bw, s), km64(bw + kSWbimg, s),
               id64, s > 0 ? 1u : 0u);
      }
      for (int s = 0; s < 8; ++s) {  // dW_layer = H_{layer-1}^T dZ_layer
        const uint64_t ah = lyr > 0 ? mn64(ain, s) : mn16(ain, s);
        const uint64_t al = lyr > 0 ? mn64(ain + kSA, s) : mn16(ain + kSA1, s);
        mma3(tmem + cw, ah, al, mn64(az, s), mn64(az + kSA, s), idT64, s > 0 ? 1u : 0u);
      }
    });
  }
  // ---- this tile's gradient row: dW from tensor memory (rows = the layer's
  // inputs: warps 0-1 hold rows 0-63), biases from the warp partials
  float* gp = grad_part + (int64_t)blockIdx.x * kMlpParams;
  if (ok) {
    if (warp < 2) {
      const int k = tid;  // layer input index
      float v[64];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + cW2 + 16 * q, v + 16 * q);
      for (int n = 0; n < 64; ++n) gp[kW2 + k * kMlpHid + n] = v[n];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + cW3 + 16 * q, v + 16 * q);
      for (int n = 0; n < 64; ++n) gp[kW3 + k * kMlpHid + n] = v[n];
      tmem_ld16(tmem + lane_off + cW4, v);
      for (int n = 0; n < kMlpOut; ++n) gp[kW4 + k * kMlpOut + n] = v[n];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(tmem + lane_off + cW1 + 16 * q, v + 16 * q);
      if (k < kMlpIn)
        for (int n = 0; n < 64; ++n) gp[kW1 + k * kMlpHid + n] = v[n];
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    l2 += __shfl_xor_sync(0xffffffffu, l2, off);
  }
  if (lane == 0) {
    sh_loss[0][warp] = l1;
    sh_loss[1][warp] = l2;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (ok) {
    for (int k = tid; k < 194; k += blockDim.x) {
      const float v = ((sDb[k] + sDb[200 + k]) + sDb[400 + k]) + sDb[600 + k];
      const int at = k < 64 ? kB1 + k : k < 128 ? kB2 + k - 64 : k < 192 ? kB3 + k - 128
                                                                        : kB4 + k - 192;
      gp[at] = v;
    }
    if (tid == 0) {
      loss_part[2 * blockIdx.x] = sh_loss[0][0] + sh_loss[0][1] + sh_loss[0][2] + sh_loss[0][3];
      loss_part[2 * blockIdx.x + 1] = sh_loss[1][0] + sh_loss[1][1] + sh_loss[1][2] + sh_loss[1][3];
    }
  } else if (tid == 0) {
    atomicOr(flags, kFlagTimeout);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// grad = sum over tiles of grad_part (fixed order)
__global__ void k_mlp_grad_reduce(int tiles, const float* __restrict__ grad_part,
                                  float* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kMlpParams; k += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int t = 0; t < tiles; ++t) s += grad_part[(int64_t)t * kMlpParams + k];
    grad[k] = s;
  }
}

// One Adam-trained batch step: fwd/bwd, weight gradients, update.
struct TrainBufs {
  float* save;
  double* loss_part;
  float* grad;
  float* m;
  float* v;
};

static gm_status grad_step(gm_ctx* c, int64_t n_data, int B, uint64_t seed, uint64_t step,
                           const float* X, const float* Y, float lam, TrainBufs& tb,
                           bool direct) {
  const int blocks = (B + 127) / 128;
  // tensor cores unless GM_MLP_TRAIN=simt (the FP32 CUDA-core kernels below)
  const char* env = std::getenv("GM_MLP_TRAIN");
  if (!(env && env[0] == 's')) {
    // tensor cores: one CTA per tile of 128 samples, then the fixed-order sum
    GM_PROF(c, "k_mlp_pack");
    k_mlp_pack<<<16, 256, 0, c->stream>>>(c->mlp_params, c->mlp_img);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_mlp_pack_bwd");
    k_mlp_pack_bwd<<<16, 256, 0, c->stream>>>(c->mlp_params, c->mlp_bimg);
    GM_LAUNCH_CHECK(c);
    cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTrainSmem);
    GM_PROF(c, "k_mlp_train_tc");
    k_mlp_train_tc<<<blocks, 128, kTrainSmem, c->stream>>>(
        n_data, B, direct ? 1 : 0, seed, step, X, Y, c->mlp_params, c->mlp_img, c->mlp_bimg, lam,
        tb.save, tb.loss_part, c->d_flags);
    GM_LAUNCH_CHECK(c);
    GM_PROF(c, "k_mlp_grad_reduce");
    k_mlp_grad_reduce<<<(kMlpParams + 255) / 256, 256, 0, c->stream>>>(blocks, tb.save, tb.grad);
    GM_LAUNCH_CHECK(c);
    return GM_OK;
  }
  const size_t smem = kMlpParams * sizeof(float);
  cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  GM_PROF(c, "k_mlp_fwd_bwd");
  // direct mode: sample s uses data row s (n_data == B)
  k_mlp_fwd_bwd<<<blocks, 128, smem, c->stream>>>(n_data, B, direct ? 1 : 0, seed, step, X, Y,
                                                  c->mlp_params, lam, tb.save, tb.loss_part);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_mlp_wgrad");
  k_mlp_wgrad<<<201, 64, 0, c->stream>>>(B, tb.save, tb.grad);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

}  // namespace gm

extern "C" gm_status gm_surrogate_grad(gm_ctx* c, int64_t n, const float* X, const float* Y,
                                       double lam, float* grad_out, double* loss_out) {
  if (!c || n < 1 || n > (1 << 20) || !X || !Y || !grad_out) return GM_E_INVAL;
  if (!c->mlp_params || !c->mlp_trained) return set_error(c, GM_E_STATE, "surrogate has no weights");
  c->launches = 0;
  const int B = (int)n;
  const int blocks = (B + 127) / 128;
  const size_t bytes = (size_t)B * kSv * sizeof(float) + (size_t)2 * blocks * sizeof(double) +
                       (size_t)kMlpParams * sizeof(float) + (size_t)B * 6 * sizeof(float);
  unsigned char* buf = (unsigned char*)dev_alloc(c, bytes);
  if (!buf) return set_error(c, GM_E_NOMEM, "gradient scratch");
  TrainBufs tb;
  tb.save = (float*)buf;
  tb.loss_part = (double*)(buf + (size_t)B * kSv * sizeof(float));
  tb.grad = (float*)(tb.loss_part + 2 * blocks);
  float* Xd = tb.grad + kMlpParams;
  float* Yd = Xd + (size_t)B * 5;
  cudaMemcpyKind kx = mlp_is_dev(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyKind ky = mlp_is_dev(Y) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(Xd, X, (size_t)B * 5 * sizeof(float), kx, c->stream));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(Yd, Y, (size_t)B * sizeof(float), ky, c->stream));
  gm_status st = grad_step(c, B, B, 0, 0, Xd, Yd, (float)lam, tb, true);
  if (st != GM_OK) return st;
  cudaMemcpyKind kg = mlp_is_dev(grad_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(grad_out, tb.grad, kMlpParams * sizeof(float), kg, c->stream));
  std::vector<double> lp(2 * blocks);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(lp.data(), tb.loss_part, lp.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  double l1 = 0, l2 = 0;
  for (int b = 0; b < blocks; ++b) {
    l1 += lp[2 * b];
    l2 += lp[2 * b + 1];
  }
  if (loss_out) *loss_out = l1 / B + lam * l2 / B;
  dev_free_now(c, buf, bytes);
  return GM_OK;
}

extern "C" gm_status gm_surrogate_train(gm_ctx* c, int64_t n_pairs, int32_t steps, int32_t batch,
                                        double lr, uint64_t seed) {
  if (!c || n_pairs < 1024 || steps < 1 || batch < 128 || batch > (1 << 18) || !(lr > 0))
    return GM_E_INVAL;
  c->launches = 0;
  gm_status st = mlp_ensure(c);
  if (st != GM_OK) return st;
  cudaStream_t s = c->stream;
  // initial parameters: He initialisation unless the context already has weights
  if (!c->mlp_trained) {
    std::vector<float> p(kMlpParams, 0.f);
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + 12345;
    auto next = [&]() {  // SplitMix64 on the host
      z += 0x9E3779B97F4A7C15ull;
      uint64_t x = z;
      x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
      x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
      return (double)((x ^ (x >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    auto gauss = [&]() {  // Box-Muller
      double u1 = std::max(next(), 1e-300), u2 = next();
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    const int fan[4] = {kMlpIn, kMlpHid, kMlpHid, kMlpHid};
    const int outs[4] = {kMlpHid, kMlpHid, kMlpHid, kMlpOut};
    const int wb[4] = {kW1, kW2, kW3, kW4};
    for (int l = 0; l < 4; ++l)
      for (int k = 0; k < fan[l] * outs[l]; ++k)
        p[wb[l] + k] = (float)(gauss() * std::sqrt(2.0 / fan[l]));
    GM_CUDA_CHECK(c, cudaMemcpy(c->mlp_params, p.data(), kMlpParams * sizeof(float),
                                cudaMemcpyHostToDevice));
  }
  // training pairs and quadrature targets
  const int64_t n = n_pairs, nv = 65536;
  const size_t dbytes = (size_t)(n + nv) * 4 * sizeof(double);
  double* dbuf = (double*)dev_alloc(c, dbytes);
  float* X = (float*)dev_alloc(c, (size_t)(n + nv) * 6 * sizeof(float));
  const int B = batch, blocks = (B + 127) / 128;
  const size_t tbytes = (size_t)B * kSv * sizeof(float) + 2 * (size_t)blocks * sizeof(double) +
                        3 * (size_t)kMlpParams * sizeof(float);
  unsigned char* tbuf = (unsigned char*)dev_alloc(c, tbytes);
  if (!dbuf || !X || !tbuf) return set_error(c, GM_E_NOMEM, "training data");
  double* si = dbuf;
  double* sj = si + (n + nv);
  double* ch = sj + (n + nv);
  double* K = ch + (n + nv);
  float* Y = X + (size_t)(n + nv) * 5;
  double* mm = (double*)c->h_pinned;
  k_minmax_s<<<1, 256, 0, s>>>(c->n, c->s, K);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(mm, K, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(s));
  const double s_min = mm[0] * 0.9, s_max = mm[1] * 1.1;
  const int gb = 8 * sm_count(c);
  // pairs like those the surrogate will serve: drawn from the neighbour pairs
  // of up to 16,384 stars spread over the catalogue; synthetic geometry only
  // if the catalogue has too few pairs
  {
    const int64_t nq = std::min<int64_t>(c->n, 16384);
    double* qbuf = (double*)dev_alloc(c, (size_t)4 * nq * sizeof(double));
    int64_t* qptr = (int64_t*)dev_alloc(c, (size_t)(nq + 1) * sizeof(int64_t));
    if (!qbuf || !qptr) return set_error(c, GM_E_NOMEM, "training pair queries");
    GM_PROF(c, "k_gather_rows");
    k_gather_rows<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nq, 256), 8 * sm_count(c))),
                    256, 0, s>>>(nq, c->n, c->s, c->ux, c->uy, c->uz, qbuf);
    GM_LAUNCH_CHECK(c);
    Buffer qcol;
    int64_t qnnz = 0;
    st = neighbour_csr(c, nq, qbuf, qbuf + nq, qbuf + 2 * nq, qbuf + 3 * nq, nullptr, false, qptr,
                       qcol, &qnnz, nullptr);
    if (st != GM_OK) return st;
    if (qnnz >= 4 * nq && qnnz >= 1024) {
      GM_PROF(c, "k_mlp_sample_cat");
      k_mlp_sample_cat<<<gb, 256, 0, s>>>(n + nv, seed, nq, qnnz, qptr, (const int32_t*)qcol.p,
                                          qbuf, qbuf + nq, qbuf + 2 * nq, qbuf + 3 * nq, c->s,
                                          c->ux, c->uy, c->uz, si, sj, ch);
    } else {
      GM_PROF(c, "k_mlp_sample");
      k_mlp_sample<<<gb, 256, 0, s>>>(n + nv, seed, s_min, s_max, c->cfg.cutoff_pc, si, sj, ch);
    }
    GM_LAUNCH_CHECK(c);
    GM_CUDA_CHECK(c, cudaStreamSynchronize(s));
    if (qcol.p) dev_free_now(c, qcol.p, qcol.bytes);
    dev_free_now(c, qptr, (size_t)(nq + 1) * sizeof(int64_t));
    dev_free_now(c, qbuf, (size_t)4 * nq * sizeof(double));
  }
  st = pairlist_quadrature(c, n + nv, si, sj, ch, K);
  if (st != GM_OK) return st;
  GM_PROF(c, "k_mlp_features");
  k_mlp_features<<<gb, 256, 0, s>>>(n + nv, si, sj, ch, K, c->cfg.sigma2, c->cfg.outer_scale_pc,
                                    X, Y);
  GM_LAUNCH_CHECK(c);
  TrainBufs tb;
  tb.save = (float*)tbuf;
  tb.loss_part = (double*)(tbuf + (size_t)B * kSv * sizeof(float));
  tb.grad = (float*)(tb.loss_part + 2 * blocks);
  tb.m = tb.grad + kMlpParams;
  tb.v = tb.m + kMlpParams;
  GM_CUDA_CHECK(c, cudaMemsetAsync(tb.m, 0, 2 * kMlpParams * sizeof(float), s));
  const float lam = 0.1f;
  double last_loss = 0;
  for (int it = 0; it < steps; ++it) {
    st = grad_step(c, n, B, seed, (uint64_t)it, X, Y, lam, tb, false);
    if (st != GM_OK) return st;
    const double frac = (double)it / steps;
    const float lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac))));
    const float c1 = (float)(1.0 - std::pow(0.9, it + 1)), c2 = (float)(1.0 - std::pow(0.999, it + 1));
    GM_PROF(c, "k_mlp_adam");
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(kMlpParams, tb.grad, c->mlp_params, tb.m,
                                                        tb.v, lr_t, 0.9f, 0.999f, c1, c2);
    GM_LAUNCH_CHECK(c);
    if (it == steps - 1) {
      std::vector<double> lp(2 * blocks);
      GM_CUDA_CHECK(c, cudaMemcpyAsync(lp.data(), tb.loss_part, lp.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(s));
      double l1 = 0, l2 = 0;
      for (int b = 0; b < blocks; ++b) {
        l1 += lp[2 * b];
        l2 += lp[2 * b + 1];
      }
      last_loss = l1 / B + lam * l2 / B;
    }
  }
  c->mlp_trained = true;
  // validation on the held-out pairs with the tensor-core network
  float* yv = (float*)tb.save;
  float* ev = yv + nv;
  MlpIn in{si + n, sj + n, ch + n, nv, c->cfg.sigma2, c->cfg.outer_scale_pc};
  st = mlp_forward(c, in, yv, ev);
  if (st != GM_OK) return st;
  std::vector<float> hy(nv), he(nv), ht(nv);
  std::vector<double> hsi(nv), hsj(nv), hch(nv);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hsi.data(), si + n, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hsj.data(), sj + n, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hch.data(), ch + n, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hy.data(), yv, nv * sizeof(float), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(he.data(), ev, nv * sizeof(float), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(ht.data(), Y + n, nv * sizeof(float), cudaMemcpyDeviceToHost, s));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(s));
  double se = 0;
  int64_t above = 0;
  for (int64_t k = 0; k < nv; ++k) {
    const double d = (double)hy[k] - (double)ht[k];
    se += d * d;
    // estimated error of the stored entry, with the taper at the pair's separation
    double w = 1.0;
    if (c->cfg.taper == GM_TAPER_WENDLAND) {
      const double dl = hsi[k] - hsj[k];
      const double h = std::sqrt(dl * dl + hsi[k] * hsj[k] * hch[k] * hch[k]) / c->cfg.cutoff_pc;
      w = h >= 1.0 ? 0.0 : std::pow(1.0 - h, 4) * (4.0 * h + 1.0);
    }
    if (w * std::exp((double)hy[k] + (double)he[k]) > c->cfg.surrogate_gate) ++above;
  }
  c->stats.surrogate_loss = last_loss;
  c->stats.surrogate_val_rmse = std::sqrt(se / nv);
  c->stats.surrogate_gate_frac = (double)above / nv;
  dev_free_now(c, tbuf, tbytes);
  dev_free_now(c, X, (size_t)(n + nv) * 6 * sizeof(float));
  dev_free_now(c, dbuf, dbytes);
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

// ---------------------------------------------------------------------------
// Covariance assembly with the surrogate: every unique pair (i <= j) of the
// neighbour CSR is evaluated by the tensor-core network; the diagonal and
// pairs whose estimated relative error exceeds the gate are recomputed by
// the sightline quadrature.
// ---------------------------------------------------------------------------
namespace gm {

__global__ void k_upper_count(int64_t n, const int64_t* __restrict__ row_ptr,
                              const int64_t* __restrict__ diag_pos, int64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = row_ptr[i + 1] - diag_pos[i];
}

__global__ void k_upper_pairs(int64_t n, const int64_t* __restrict__ diag_pos,
                              const int32_t* __restrict__ col, const int64_t* __restrict__ uptr,
                              const double* __restrict__ s, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ uz,
                              int64_t* __restrict__ pe, int32_t* __restrict__ prow,
                              double* __restrict__ psi, double* __restrict__ psj,
                              double* __restrict__ pch, double* __restrict__ pdist) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t p0 = uptr[i], cnt = uptr[i + 1] - p0, e0 = diag_pos[i];
    for (int64_t t = lane; t < cnt; t += 32) {
      const int64_t e = e0 + t, p = p0 + t;
      const int32_t j = col[e];
      const double dx = ux[i] - ux[j], dy = uy[i] - uy[j], dz = uz[i] - uz[j];
      const double c2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double ds = s[i] - s[j];
      pe[p] = e;
      prow[p] = (int32_t)i;
      psi[p] = s[i];
      psj[p] = s[j];
      pch[p] = sqrt(c2);
      pdist[p] = sqrt(fma(ds, ds, s[i] * s[j] * c2));
    }
  }
}

__device__ __forceinline__ double taper_w(double h) {
  if (h >= 1.0) return 0.0;
  const double u = 1.0 - h, u2 = u * u;
  return u2 * u2 * (4.0 * h + 1.0);
}

template <typename T>
__global__ void k_surrogate_apply(int64_t np, const int64_t* __restrict__ pe,
                                  const int32_t* __restrict__ prow, const int32_t* __restrict__ col,
                                  const double* __restrict__ pdist, const float* __restrict__ y,
                                  const float* __restrict__ e, double gate, double inv_cut,
                                  int taper, T* __restrict__ val, int64_t* __restrict__ flag) {
  const double loggate = log(gate);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ee = pe[p];
    const bool diag = col[ee] == prow[p];
    const float yp = y[p], ep = e[p];
    // estimated absolute error of the stored (tapered) entry:
    // W K |y - y_true| = W exp(y + e)
    const double w = taper == GM_TAPER_WENDLAND ? taper_w(pdist[p] * inv_cut) : 1.0;
    const bool fb = diag || !isfinite(yp) || !isfinite(ep) ||
                    !((double)yp + (double)ep + log(w) <= loggate);
    flag[p] = fb ? 1 : 0;
    if (!fb) val[ee] = (T)(w * exp((double)yp));
  }
}

__global__ void k_fallback_gather(int64_t np, const int64_t* __restrict__ flag,
                                  const int64_t* __restrict__ pos, const double* __restrict__ psi,
                                  const double* __restrict__ psj, const double* __restrict__ pch,
                                  int64_t* __restrict__ fl, double* __restrict__ fsi,
                                  double* __restrict__ fsj, double* __restrict__ fch) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (flag[p]) {
      const int64_t q = pos[p];
      fl[q] = p;
      fsi[q] = psi[p];
      fsj[q] = psj[p];
      fch[q] = pch[p];
    }
  }
}

template <typename T>
__global__ void k_fallback_write(int64_t nf, const int64_t* __restrict__ fl,
                                 const int64_t* __restrict__ pe, const int32_t* __restrict__ prow,
                                 const int32_t* __restrict__ col, const double* __restrict__ pdist,
                                 const double* __restrict__ psi, const double* __restrict__ K,
                                 double inv_cut, int taper, int form, double log_rho_bar,
                                 double sigma2, T* __restrict__ val, double* __restrict__ kdiag,
                                 double* __restrict__ prior_m, unsigned* __restrict__ flags) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nf;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = fl[q], ee = pe[p];
    const int32_t i = prow[p];
    double Kv = K[q];
    if (!isfinite(Kv)) atomicOr(flags, kFlagNonFinite);
    if (col[ee] == i) {
      val[ee] = (T)Kv;
      kdiag[i] = (double)(T)Kv;
      prior_m[i] = log_rho_bar + log(psi[p]) -
                   (form == GM_FORM_LOGNORMAL ? 0.5 * (double)(T)Kv : 0.5 * sigma2);
    } else {
      if (taper == GM_TAPER_WENDLAND) Kv *= taper_w(pdist[p] * inv_cut);
      val[ee] = (T)Kv;
    }
  }
}

template <typename T>
static gm_status surrogate_values_t(gm_ctx* c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->n;
  const int sms = sm_count(c);
  int64_t* cnt = (int64_t*)dev_alloc(c, (n + 1) * sizeof(int64_t));
  int64_t* uptr = (int64_t*)dev_alloc(c, (n + 1) * sizeof(int64_t));
  if (!cnt || !uptr) return set_error(c, GM_E_NOMEM, "surrogate pair list");
  const int eb = (int)std::min<int64_t>(ceil_div(n, 256), 8 * sms);
  GM_PROF(c, "k_upper_count");
  k_upper_count<<<eb, 256, 0, st>>>(n, c->row_ptr, c->diag_pos, cnt);
  GM_LAUNCH_CHECK(c);
  gm_status s = scan_i64(c, cnt, uptr, n);
  if (s != GM_OK) return s;
  int64_t np = 0;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(&np, uptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  // per pair: pe, flag, pos (int64), prow (int32), si, sj, chord, dist (double), y, e (float)
  const size_t per = 3 * 8 + 4 + 4 * 8 + 2 * 4;
  const size_t bytes = (size_t)(np + 1) * per + 64;
  unsigned char* buf = (unsigned char*)dev_alloc(c, bytes);
  if (!buf) return set_error(c, GM_E_NOMEM, "surrogate pair list");
  int64_t* pe = (int64_t*)buf;
  int64_t* flag = pe + (np + 1);
  int64_t* pos = flag + (np + 1);
  double* psi = (double*)(pos + (np + 1));
  double* psj = psi + (np + 1);
  double* pch = psj + (np + 1);
  double* pdist = pch + (np + 1);
  int32_t* prow = (int32_t*)(pdist + (np + 1));
  float* y = (float*)(prow + (np + 1));
  float* e = y + (np + 1);
  const int wb = (int)std::min<int64_t>(ceil_div(n * 32, 256), 16 * sms);
  GM_PROF(c, "k_upper_pairs");
  k_upper_pairs<<<wb, 256, 0, st>>>(n, c->diag_pos, c->col, uptr, c->s, c->ux, c->uy, c->uz, pe,
                                    prow, psi, psj, pch, pdist);
  GM_LAUNCH_CHECK(c);
  MlpIn in{psi, psj, pch, np, c->cfg.sigma2, c->cfg.outer_scale_pc};
  s = mlp_forward(c, in, y, e);
  if (s != GM_OK) return s;
  const int pb = (int)std::min<int64_t>(ceil_div(np, 256), 16 * sms);
  const double inv_cut = 1.0 / c->cfg.cutoff_pc;
  GM_PROF(c, "k_surrogate_apply");
  k_surrogate_apply<T><<<pb, 256, 0, st>>>(np, pe, prow, c->col, pdist, y, e, c->cfg.surrogate_gate,
                                           inv_cut, c->cfg.taper, (T*)c->val, flag);
  GM_LAUNCH_CHECK(c);
  s = scan_i64(c, flag, pos, np);
  if (s != GM_OK) return s;
  int64_t nf = 0;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(&nf, pos + np, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  const size_t fbytes = (size_t)(nf + 1) * (8 + 4 * 8);
  unsigned char* fbuf = (unsigned char*)dev_alloc(c, fbytes);
  if (!fbuf) return set_error(c, GM_E_NOMEM, "surrogate fallback list");
  int64_t* fl = (int64_t*)fbuf;
  double* fsi = (double*)(fl + (nf + 1));
  double* fsj = fsi + (nf + 1);
  double* fch = fsj + (nf + 1);
  double* fK = fch + (nf + 1);
  GM_PROF(c, "k_fallback_gather");
  k_fallback_gather<<<pb, 256, 0, st>>>(np, flag, pos, psi, psj, pch, fl, fsi, fsj, fch);
  GM_LAUNCH_CHECK(c);
  s = pairlist_quadrature(c, nf, fsi, fsj, fch, fK);
  if (s != GM_OK) return s;
  const int fb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nf, 256), 16 * sms));
  GM_PROF(c, "k_fallback_write");
  k_fallback_write<T><<<fb, 256, 0, st>>>(nf, fl, pe, prow, c->col, pdist, psi, fK, inv_cut,
                                          c->cfg.taper, c->cfg.form, std::log(c->cfg.rho_bar),
                                          c->cfg.sigma2, (T*)c->val, c->kdiag, c->prior_m,
                                          c->d_flags);
  GM_LAUNCH_CHECK(c);
  s = mirror_csr(c, n, c->row_ptr, c->col, c->nnz, c->val);
  if (s != GM_OK) return s;
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  c->stats.surrogate_fallback = nf - n;  // the n diagonal entries always use the quadrature
  dev_free_now(c, fbuf, fbytes);
  dev_free_now(c, buf, bytes);
  dev_free_now(c, uptr, (n + 1) * sizeof(int64_t));
  dev_free_now(c, cnt, (n + 1) * sizeof(int64_t));
  return GM_OK;
}

gm_status surrogate_values(gm_ctx* c) {
  if (!c->mlp_trained) return set_error(c, GM_E_STATE, "surrogate source selected but not trained");
  if (c->n_fields > 1) return set_error(c, GM_E_STATE, "surrogate needs a single-field context");
  if (c->cfg.precision == GM_PREC_FP32) return surrogate_values_t<float>(c);
  return surrogate_values_t<double>(c);
}

}  // namespace gm

// ---------------------------------------------------------------------------
// Streamed assembly of a block of rows (gm_cov_rows).  A catalogue whose
// covariance does not fit in memory (the 1,000,000-star field: ~3.7e10
// stored entries) is assembled block by block: the neighbour rows of stars
// row0 .. row0 + nrows - 1 (internal order) against all stars, with values by
// the quadrature or by the surrogate with the quadrature at the gate, as
// gm_build_cov computes them (the taper applied; the diagonal always by the
// quadrature).
// ---------------------------------------------------------------------------
namespace gm {

__global__ void k_chunk_pairs(int64_t nrows, int64_t row0, const int64_t* __restrict__ qptr,
                              const int32_t* __restrict__ qcol, const double* __restrict__ s,
                              const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ uz, double* __restrict__ psi,
                              double* __restrict__ psj, double* __restrict__ pch,
                              double* __restrict__ pdist, int32_t* __restrict__ pdiag) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < nrows; r += nw) {
    const int64_t i = row0 + r;
    for (int64_t e = qptr[r] + lane; e < qptr[r + 1]; e += 32) {
      const int32_t j = qcol[e];
      const double dx = ux[i] - ux[j], dy = uy[i] - uy[j], dz = uz[i] - uz[j];
      const double c2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double ds = s[i] - s[j];
      psi[e] = s[i];
      psj[e] = s[j];
      pch[e] = sqrt(c2);
      pdist[e] = sqrt(fma(ds, ds, s[i] * s[j] * c2));
      pdiag[e] = j == i;
    }
  }
}

template <typename T>
__global__ void k_chunk_apply(int64_t np, const int32_t* __restrict__ pdiag,
                              const double* __restrict__ pdist, const float* __restrict__ y,
                              const float* __restrict__ e, double gate, double inv_cut, int taper,
                              T* __restrict__ val, int64_t* __restrict__ flag) {
  const double loggate = log(gate);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float yp = y[p], ep = e[p];
    const double w = taper == GM_TAPER_WENDLAND ? taper_w(pdist[p] * inv_cut) : 1.0;
    const bool fb = pdiag[p] || !isfinite(yp) || !isfinite(ep) ||
                    !((double)yp + (double)ep + log(w) <= loggate);
    flag[p] = fb ? 1 : 0;
    if (!fb) val[p] = (T)(w * exp((double)yp));
  }
}

template <typename T>
__global__ void k_chunk_fallback(int64_t nf, const int64_t* __restrict__ fl,
                                 const int32_t* __restrict__ pdiag,
                                 const double* __restrict__ pdist, const double* __restrict__ K,
                                 double inv_cut, int taper, T* __restrict__ val,
                                 unsigned* __restrict__ flags) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nf;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = fl[q];
    double Kv = K[q];
    if (!isfinite(Kv)) atomicOr(flags, kFlagNonFinite);
    if (!pdiag[p] && taper == GM_TAPER_WENDLAND) Kv *= taper_w(pdist[p] * inv_cut);
    val[p] = (T)Kv;
  }
}

template <typename T>
static gm_status cov_rows_t(gm_ctx* c, int64_t row0, int64_t nrows, int32_t source,
                            int64_t* rp_out, int32_t* col_out, void* val_out, int64_t cap,
                            int64_t* nnz_out, int64_t* fallback_out) {
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  ScopedDev bqp(c, (size_t)(nrows + 1) * sizeof(int64_t));
  int64_t* qptr = (int64_t*)bqp.p;
  if (!qptr) return set_error(c, GM_E_NOMEM, "row-block pointers");
  Buffer qcol;
  int64_t nnz = 0;
  gm_status s = neighbour_csr(c, nrows, c->s + row0, c->ux + row0, c->uy + row0, c->uz + row0,
                              nullptr, false, qptr, qcol, &nnz, nullptr);
  if (s != GM_OK) return s;
  ScopedDev bqc(c, qcol.p, qcol.bytes, ScopedDev::Adopt{});
  *nnz_out = nnz;
  if (fallback_out) *fallback_out = 0;
  if (nnz > cap) return set_error(c, GM_E_INVAL, "row block: more entries than the capacity");
  ScopedDev bval(c, (size_t)std::max<int64_t>(nnz, 1) * sizeof(T));
  T* val = (T*)bval.p;
  if (!val) return set_error(c, GM_E_NOMEM, "row-block values");
  if (source == GM_COV_QUADRATURE || nnz == 0) {
    s = pair_quadrature(c, nrows, c->s + row0, c->ux + row0, c->uy + row0, c->uz + row0, nullptr,
                        qptr, (const int32_t*)qcol.p, nnz, val, false);
    if (s != GM_OK) return s;
  } else {
    // per entry: si, sj, chord, distance (double), diagonal (int32), y, e
    // (float), flag, position (int64)
    const size_t per = 4 * 8 + 4 + 2 * 4 + 2 * 8;
    ScopedDev bp(c, (size_t)(nnz + 1) * per + 64);
    if (!bp.p) return set_error(c, GM_E_NOMEM, "row-block pair list");
    double* psi = (double*)bp.p;
    double* psj = psi + (nnz + 1);
    double* pch = psj + (nnz + 1);
    double* pdist = pch + (nnz + 1);
    int64_t* flag = (int64_t*)(pdist + (nnz + 1));
    int64_t* pos = flag + (nnz + 1);
    float* y = (float*)(pos + (nnz + 1));
    float* e = y + (nnz + 1);
    int32_t* pdiag = (int32_t*)(e + (nnz + 1));
    const int wb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nrows * 32, 256), 16 * sms));
    GM_PROF(c, "k_chunk_pairs");
    k_chunk_pairs<<<wb, 256, 0, st>>>(nrows, row0, qptr, (const int32_t*)qcol.p, c->s, c->ux,
                                      c->uy, c->uz, psi, psj, pch, pdist, pdiag);
    GM_LAUNCH_CHECK(c);
    MlpIn in{psi, psj, pch, nnz, c->cfg.sigma2, c->cfg.outer_scale_pc};
    s = mlp_forward(c, in, y, e);
    if (s != GM_OK) return s;
    const int pb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nnz, 256), 16 * sms));
    GM_PROF(c, "k_chunk_apply");
    k_chunk_apply<T><<<pb, 256, 0, st>>>(nnz, pdiag, pdist, y, e, c->cfg.surrogate_gate,
                                         1.0 / c->cfg.cutoff_pc, c->cfg.taper, val, flag);
    GM_LAUNCH_CHECK(c);
    s = scan_i64(c, flag, pos, nnz);
    if (s != GM_OK) return s;
    int64_t nf = 0;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(&nf, pos + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
    ScopedDev bf(c, (size_t)(nf + 1) * (8 + 4 * 8));
    if (!bf.p) return set_error(c, GM_E_NOMEM, "row-block fallback list");
    int64_t* fl = (int64_t*)bf.p;
    double* fsi = (double*)(fl + (nf + 1));
    double* fsj = fsi + (nf + 1);
    double* fch = fsj + (nf + 1);
    double* fK = fch + (nf + 1);
    GM_PROF(c, "k_fallback_gather");
    k_fallback_gather<<<pb, 256, 0, st>>>(nnz, flag, pos, psi, psj, pch, fl, fsi, fsj, fch);
    GM_LAUNCH_CHECK(c);
    s = pairlist_quadrature(c, nf, fsi, fsj, fch, fK);
    if (s != GM_OK) return s;
    GM_PROF(c, "k_chunk_fallback");
    k_chunk_fallback<T><<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nf, 256), 16 * sms)),
                          256, 0, st>>>(nf, fl, pdiag, pdist, fK, 1.0 / c->cfg.cutoff_pc,
                                        c->cfg.taper, val, c->d_flags);
    GM_LAUNCH_CHECK(c);
    if (fallback_out) *fallback_out = nf;
  }
  // results to the caller (host or device)
  GM_CUDA_CHECK(c, cudaMemcpyAsync(rp_out, qptr, (size_t)(nrows + 1) * sizeof(int64_t),
                                   cudaMemcpyDefault, st));
  if (nnz > 0) {
    GM_CUDA_CHECK(c, cudaMemcpyAsync(col_out, qcol.p, (size_t)nnz * sizeof(int32_t),
                                     cudaMemcpyDefault, st));
    GM_CUDA_CHECK(c, cudaMemcpyAsync(val_out, val, (size_t)nnz * sizeof(T), cudaMemcpyDefault,
                                     st));
  }
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  return GM_OK;
}

}  // namespace gm

extern "C" gm_status gm_cov_rows(gm_ctx* c, int64_t row0, int64_t nrows, int32_t source,
                                 int64_t capacity, int64_t* row_ptr_out, int32_t* col_out,
                                 void* val_out, int64_t* nnz_out, int64_t* fallback_out) {
  if (!c || row0 < 0 || nrows < 1 || row0 + nrows > c->n || capacity < 0 || !row_ptr_out ||
      !nnz_out || (capacity > 0 && (!col_out || !val_out)))
    return GM_E_INVAL;
  if (source != GM_COV_QUADRATURE && source != GM_COV_SURROGATE) return GM_E_INVAL;
  if (c->n_fields > 1) return set_error(c, GM_E_STATE, "row blocks need a single-field context");
  if (source == GM_COV_SURROGATE && !c->mlp_trained)
    return set_error(c, GM_E_STATE, "surrogate source selected but not trained");
  c->launches = 0;
  gm_status st = c->cfg.precision == GM_PREC_FP32
                     ? cov_rows_t<float>(c, row0, nrows, source, row_ptr_out, col_out, val_out,
                                         capacity, nnz_out, fallback_out)
                     : cov_rows_t<double>(c, row0, nrows, source, row_ptr_out, col_out, val_out,
                                          capacity, nnz_out, fallback_out);
  if (st == GM_OK) st = read_flags(c);
  prof_collect(c);
  c->stats.kernel_launches = c->launches;
  return st;
}
