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

// tanh x = (e^{2x} - 1) / (e^{2x} + 1) with the hardware base-2 exponential
// (e^{2x} = 2^{2x log2 e}) and reciprocal.  |x| is clamped to 9, where
// tanh differs from +-1 by less than half an FP32 ulp of 1.  The absolute
// error is a few 1e-8 (relative error grows only for |x| << 1e-6, where the
// result is below the rounding noise of the dot products it feeds).
__device__ __forceinline__ float tanh_f32(float x) {
  const float xc = fminf(fmaxf(x, -9.0f), 9.0f);
  const float e = ex2_approx(xc * 2.8853900817779268f);
  return (e - 1.0f) * rcp_approx(e + 1.0f);
}

__device__ __forceinline__ float activation(float a, int act) { return act == 1 ? a : tanh_f32(a); }

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
