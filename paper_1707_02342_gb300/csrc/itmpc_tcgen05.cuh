// itmpc_tcgen05.cuh -- inline-PTX wrappers for the 5th-generation tensor cores
// (tcgen05: MMA from shared-memory descriptors into tensor memory, TMEM
// allocation, TMEM -> register loads) used by the reduced-precision rollout.
//
// Shared-memory operand layout: K-major without swizzle, built from
// "core matrices" of 8 rows x 16 bytes stored as 128 contiguous bytes.  For an
// R x Kb-byte tile, byte kb of row r lives at
//     (r / 8) * (Kb * 8) + (kb / 16) * 128 + (r % 8) * 16 + kb % 16,
// so the leading-dimension byte offset (next core matrix along K) is 128 and
// the stride-dimension byte offset (next group of 8 rows) is Kb * 8.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace itmpc {

__host__ __device__ constexpr int cm_offset(int r, int kb, int Kb) {
  return (r >> 3) * (Kb * 8) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, dense, FP32 accumulator, both operands K-major.
// bf16: A and B BF16 (kind::f16); otherwise A and B E4M3 (kind::f8f6f4).
__host__ __device__ constexpr uint32_t tc_idesc(bool bf16, int M, int N) {
  return (1u << 4) | (bf16 ? ((1u << 7) | (1u << 10)) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tc_mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Same with the A operand in tensor memory: lane r = row r, each 32-bit column packs
// consecutive K elements (2 BF16 or 4 E4M3, lowest first); one 32-byte K-step = 8 columns.
__device__ __forceinline__ void tc_mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tc_mma_e4m3_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

// The mbarrier receives one arrival once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(mbar))
               : "memory");
}

// Whole warp: allocate `ncols` TMEM columns (power of two >= 32); the base address goes to *slot.
__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Warp loads 32 consecutive FP32 columns of its 32 TMEM lanes (lane i -> thread i).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// Warp stores 2 / 4 / 8 consecutive 32-bit columns of its 32 TMEM lanes (thread i -> lane i).
__device__ __forceinline__ void tc_st2(uint32_t taddr, uint32_t a, uint32_t b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(a), "r"(b) : "memory");
}

__device__ __forceinline__ void tc_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

__device__ __forceinline__ void tc_st8(uint32_t taddr, uint4 lo, uint4 hi) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(lo.x), "r"(lo.y), "r"(lo.z), "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
               : "memory");
}

// This thread's earlier tcgen05.st have completed.
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Hardware tanh (MUFU), ~2^-11 relative error: below the BF16/E4M3 rounding it feeds.
__device__ __forceinline__ float tanh_mufu(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tanh on the FMA pipe, for the share of an epilogue's activations that would otherwise
// queue behind the MUFU unit (15 results per clock per SM):  tanh(x) ~ c q(|c|),
// c = x clamped to [-4.3, 4.3] (NaN kept), q a degree-8 polynomial fitted to tanh(y)/y on
// [0, 4.3] by iteratively reweighted least squares on Chebyshev points.  Evaluated in FP32
// by Horner's rule, |error| <= 2.4e-4 for every input (tanh(4.3) = 1 - 3.7e-4): inside the
// hardware tanh's own bound (2^-10.99 relative, |tanh| <= 1) and far below the BF16 rounding
// (2^-9 relative) of the operand it feeds.  11 instructions, odd: tanh(0) = 0 exactly.
constexpr float kTanhPolyClamp = 4.3f;
__device__ __forceinline__ float tanh_poly(float x) {
  constexpr float kTanhPoly[9] = {9.930922389e-01f, 6.841585040e-02f, -5.574090481e-01f,
                                  3.255223334e-01f, -6.596770883e-02f, -6.843555719e-03f,
                                  5.668960977e-03f, -9.846792091e-04f, 5.915315342e-05f};
  float c;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(c) : "f"(x), "f"(-kTanhPolyClamp));
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(c) : "f"(c), "f"(kTanhPolyClamp));
  const float y = fabsf(c);
  float q = kTanhPoly[8];
#pragma unroll
  for (int k = 7; k >= 0; --k) q = fmaf(q, y, kTanhPoly[k]);
  return c * q;
}

}  // namespace itmpc
