// Small inline-PTX helpers for the 5th-generation tensor cores (tcgen05),
// mbarriers and bulk copies, shared by the tensor-core kernels of the
// deflated preconditioner.  sm_100-family only.
#pragma once
#include <cstdint>

namespace gm {
namespace tg {

__device__ __forceinline__ uint32_t smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version bit, layout (0 = no swizzle,
// 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                         uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, M x N; a_mn / b_mn
// select the MN-major (transposed) layout of A / B.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B (+ D when acc != 0), issued by one thread
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// the mbarrier completes its phase when every earlier MMA of this thread is done
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) completing on an mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(mbar)
      : "memory");
}

// Bounded wait on an mbarrier phase: false when it gave up (after about 2^26
// polls) or when another thread raised *abort.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity, volatile int* abort) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && (it & 255u) == 255u && *abort) return false;
  }
  return false;
}

// 16 consecutive FP32 columns of the warp's 32 tensor-memory lanes
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&u)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x rounded to BF16 (nearest, ties to even) as an FP32 bit pattern with zero
// low half, by integer arithmetic on the bits
__device__ __forceinline__ uint32_t rne_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// three BF16 pieces of x: x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
__device__ __forceinline__ void split3(float x, uint32_t& a, uint32_t& b, uint32_t& c) {
  a = rne_bits(x);
  const float r1 = x - __uint_as_float(a);
  b = rne_bits(r1);
  const float r2 = r1 - __uint_as_float(b);
  c = rne_bits(r2);
}

// BF16 values (high halves of lo and hi) in one word, lo first
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x7632);
}

// eight FP32 values -> three 16-byte rows of BF16 pieces
__device__ __forceinline__ void split3x8(const float* v, uint4& p1, uint4& p2, uint4& p3) {
  uint32_t a[8], b[8], c[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) split3(v[e], a[e], b[e], c[e]);
  p1 = make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
  p2 = make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
  p3 = make_uint4(pack2(c[0], c[1]), pack2(c[2], c[3]), pack2(c[4], c[5]), pack2(c[6], c[7]));
}

// four FP32 values -> three 8-byte rows of BF16 pieces
__device__ __forceinline__ void split3x4(const float* v, uint2& p1, uint2& p2, uint2& p3) {
  uint32_t a[4], b[4], c[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) split3(v[e], a[e], b[e], c[e]);
  p1 = make_uint2(pack2(a[0], a[1]), pack2(a[2], a[3]));
  p2 = make_uint2(pack2(b[0], b[1]), pack2(b[2], b[3]));
  p3 = make_uint2(pack2(c[0], c[1]), pack2(c[2], c[3]));
}

}  // namespace tg
}  // namespace gm
