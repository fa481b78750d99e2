// itmpc_device.cuh -- device building blocks of the IT-MPC iteration (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "itmpc_internal.h"

namespace itmpc {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 (hi/lo halves) and
// mixes in the key, which is bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Box-Muller on u_i = ((w_i >> 8) + 1) 2^-24 in (0, 1], exact in binary32.
__device__ __forceinline__ float2 box_muller(uint32_t a0, uint32_t a1) {
  const float u0 = __uint2float_rn((a0 >> 8) + 1u) * 5.9604644775390625e-8f;
  const float u1 = __uint2float_rn((a1 >> 8) + 1u) * 5.9604644775390625e-8f;
  const float r = sqrtf(-2.0f * logf(u0));
  float s, c;
  sincospif(2.0f * u1, &s, &c);  // sin(2 pi u1), cos(2 pi u1)
  return make_float2(r * c, r * s);
}

// eps_{k,t} = (sigma_0 z0, sigma_1 z1) with counter (k, t, ctr2, ctr3).
__device__ __forceinline__ float2 noise_at(const IterParams &p, uint32_t k, uint32_t t) {
  const uint4 w = philox4x32_10(make_uint4(k, t, p.ctr2, p.ctr3), p.key0, p.key1);
  const float2 z = box_muller(w.x, w.y);
  return make_float2(p.sigma0 * z.x, p.sigma1 * z.y);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tanh x = 1 - 2 / (1 + e^{2x}), with e^{2x} = 2^{2x log2 e} from the hardware
// base-2 exponential and the division from the hardware reciprocal.  Both ends
// saturate without a clamp: e^{2x} = +inf gives 1 - 2/inf = 1 and e^{2x} -> 0
// gives 1 - 2 = -1.  Near 0 the subtraction cancels, leaving an absolute error
// of about two FP32 ulps of 1 -- below the rounding noise of the dot products
// the activation feeds.
__device__ __forceinline__ float tanh_f32(float x) {
  const float e = ex2_approx(x * 2.8853900817779268f);
  return fmaf(-2.0f, rcp_approx(1.0f + e), 1.0f);
}

// ---- packed FP32 pairs (sm_100+ fma.rn.f32x2: two IEEE FMAs per instruction) ----
__device__ __forceinline__ unsigned long long f2pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}

__device__ __forceinline__ float2 f2unpack(unsigned long long r) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
  return make_float2(x, y);
}

// (a.x b.x + c.x, a.y b.y + c.y), each rounded once as by fmaf
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int ACT>
__device__ __forceinline__ float activation(float a) {
  if constexpr (ACT == 1) return a;
  else return tanh_f32(a);
}

// h(p_x, p_y): bilinear, texel (i, j) centred at origin + (j + 1/2, i + 1/2) res,
// clamp-to-edge.  NaN positions give NaN (indices stay in range).
__device__ __forceinline__ float costmap_h(const IterParams &p, float px, float py) {
  const float fx = (px - p.origin_x) * p.inv_res - 0.5f;
  const float fy = (py - p.origin_y) * p.inv_res - 0.5f;
  const float jf = floorf(fx), if_ = floorf(fy);
  const float a = fx - jf, b = fy - if_;
  const float jc = fminf(fmaxf(jf, -1.0f), (float)p.map_w);
  const float ic = fminf(fmaxf(if_, -1.0f), (float)p.map_h);
  const int jj = (int)jc, ii = (int)ic;
  const int j0 = min(max(jj, 0), p.map_w - 1), j1 = min(max(jj + 1, 0), p.map_w - 1);
  const int i0 = min(max(ii, 0), p.map_h - 1), i1 = min(max(ii + 1, 0), p.map_h - 1);
  const float *r0 = p.map + (size_t)i0 * p.map_w;
  const float *r1 = p.map + (size_t)i1 * p.map_w;
  const float m00 = __ldg(r0 + j0), m01 = __ldg(r0 + j1);
  const float m10 = __ldg(r1 + j0), m11 = __ldg(r1 + j1);
  return (1.0f - a) * (1.0f - b) * m00 + a * (1.0f - b) * m01 + (1.0f - a) * b * m10 + a * b * m11;
}

// State cost at loop index t (1..T): Sec. V-C track + speed + stabilizing terms.
__device__ __forceinline__ float state_cost(const IterParams &p, float px, float py, float vx, float vy, int t) {
  float h = costmap_h(p, px, py);
  h = h > p.map_cap ? p.map_cap : h;  // NaN stays NaN
  const float zeta = -atan2f(vy, fabsf(vx));
  const float sp = vx - p.v_des;
  float imp = 0.0f;
  if (h > p.track_thresh) imp += exp2f((float)t * p.log2_decay) * p.crash_cost;
  if (fabsf(zeta) > p.slip_thresh) imp += p.crash_cost;
  return p.w_track * h + p.w_speed * sp * sp + p.w_stab * zeta * zeta + p.w_crash * imp;
}

// ---- asynchronous bulk copies (cp.async.bulk) completed on an mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival (release at CTA scope: the arriving thread's earlier shared-memory writes,
// and those a __syncwarp ordered before it, are visible to a thread whose wait sees the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// Prefetch `bytes` (multiple of 16) at a 16-byte aligned global address into L2.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// 4-byte asynchronous global -> shared copy (cp.async; completion by cp_async_wait_all of the
// same thread): the value lands in shared memory without occupying a register meanwhile.
__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Order this thread's earlier generic-proxy accesses before later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

template <typename F>
__device__ __forceinline__ float warp_reduce(float v, F op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(FULL_MASK, v, o));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
  return warp_reduce(v, [](float a, float b) { return a + b; });
}
__device__ __forceinline__ float warp_min(float v) {
  return warp_reduce(v, [](float a, float b) { return fminf(a, b); });
}

__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float n = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

}  // namespace itmpc
