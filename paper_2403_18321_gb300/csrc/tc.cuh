// tc.cuh -- tcgen05 (5th-generation tensor core) helpers shared by the
// tensor-core kernels: fences, the shared-memory operand and instruction
// descriptors of kind::f16 (FP16 operands, FP32 accumulation in TMEM), MMA
// issue and commit, TMEM loads, and the FP16 pair conversions of the
// two-term split x = hi + lo.
#pragma once

#include "tma.cuh"

namespace gbpca {

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory operand descriptor, K-major, no swizzle: core matrix = 8 rows
// x 16 bytes; lbo = byte stride between K-adjacent core matrices, sbo =
// between 8-row groups.
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Shared-memory operand descriptor, K-major with the 128-byte swizzle: rows of
// 128 bytes (64 FP16 K-values), the 16-byte units of row r stored at unit
// index u ^ (r mod 8), 8-row groups 1024 bytes apart (the atom must be 1024-byte
// aligned).  A K-step of 16 values inside the atom adds 32 bytes to the start.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}
// kind::f16 instruction descriptor: D F32, A/B F16 (format 0), both K-major,
// M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// The same two, executed by a whole warp (convergent control flow keeps the
// descriptors in uniform registers); one elected lane issues the instruction.
__device__ __forceinline__ void mma_f16_warp(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit_warp(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
          su32(bar))
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads (e.g. of two accumulators) in flight, one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  uint32_t r;  // low half = a, high half = b
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ void unpack_f16x2(uint32_t v, float& a, float& b) {
  a = __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
  b = __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}

// x = y s + c for a packed BF16 pair y (low half first) and packed BF16 scales
// s, with FP32 c and results: the product is exact (the scales are powers of
// two), the sum rounded once -- fmaf on the widened operands, without them.
__device__ __forceinline__ void fma_bf16x2_f32(uint32_t y, uint32_t s, float c0, float c1,
                                               float& x0, float& x1) {
  asm("{\n .reg .b16 y0, y1, s0, s1;\n mov.b32 {y0, y1}, %2;\n mov.b32 {s0, s1}, %3;\n"
      " fma.rn.f32.bf16 %0, y0, s0, %4;\n fma.rn.f32.bf16 %1, y1, s1, %5;\n}"
      : "=f"(x0), "=f"(x1)
      : "r"(y), "r"(s), "f"(c0), "f"(c1));
}
// r = x - hi for a packed FP16 pair hi (low half first): exact, since hi is x
// rounded to FP16.
__device__ __forceinline__ void resid_f16x2(uint32_t hi, float x0, float x1, float& r0,
                                            float& r1) {
  asm("{\n .reg .b16 h0, h1, m;\n mov.b32 {h0, h1}, %2;\n mov.b16 m, 0xbc00;\n"
      " fma.rn.f32.f16 %0, h0, m, %3;\n fma.rn.f32.f16 %1, h1, m, %4;\n}"
      : "=f"(r0), "=f"(r1)
      : "r"(hi), "f"(x0), "f"(x1));
}
// Whether either half of a packed FP16 pair is an infinity.  When x leaves
// the FP16 range, hi = fp16(x) is an infinity and so is lo = fp16(x - hi).
__device__ __forceinline__ bool f16x2_has_inf(uint32_t v) {
  const uint32_t a = v & 0x7fff7fffu;
  return (a & 0xffffu) == 0x7c00u || (a >> 16) == 0x7c00u;
}
// The same for a packed FP16 pair y and packed FP16 scales s.
__device__ __forceinline__ void fma_f16x2_f32(uint32_t y, uint32_t s, float c0, float c1,
                                              float& x0, float& x1) {
  asm("{\n .reg .b16 y0, y1, s0, s1;\n mov.b32 {y0, y1}, %2;\n mov.b32 {s0, s1}, %3;\n"
      " fma.rn.f32.f16 %0, y0, s0, %4;\n fma.rn.f32.f16 %1, y1, s1, %5;\n}"
      : "=f"(x0), "=f"(x1)
      : "r"(y), "r"(s), "f"(c0), "f"(c1));
}
// FP16 bits of 2^e (-14 <= e <= 15: the normal range)
__device__ __forceinline__ uint32_t f16_pow2(int e) { return (uint32_t)(e + 15) << 10; }
// BF16 bits of 2^e (|e| <= 126)
__device__ __forceinline__ uint32_t bf16_pow2(int e) { return (uint32_t)(e + 127) << 7; }


}  // namespace gbpca
