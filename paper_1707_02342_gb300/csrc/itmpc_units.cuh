// itmpc_units.cuh -- per-sample device steps shared by the kernels that work
// on 128-sample units of possibly many instances (TpsShared parameters).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_internal.h"

namespace itmpc {

__device__ __forceinline__ float2 tps_noise(const TpsShared &sh, uint32_t k, uint32_t t, uint32_t c2, uint32_t c3) {
  const uint4 w = philox4x32_10(make_uint4(k, t, c2, c3), sh.key0, sh.key1);
  const float2 z = box_muller(w.x, w.y);
  return make_float2(sh.sigma0 * z.x, sh.sigma1 * z.y);
}

// h(p_x, p_y): bilinear, texel (i, j) centred at origin + (j + 1/2, i + 1/2) res, clamp-to-edge.
__device__ __forceinline__ float tps_costmap(const TpsShared &sh, const float *map, float px, float py) {
  const float fx = (px - sh.origin_x) * sh.inv_res - 0.5f;
  const float fy = (py - sh.origin_y) * sh.inv_res - 0.5f;
  const float jf = floorf(fx), if_ = floorf(fy);
  const float a = fx - jf, b = fy - if_;
  const float jc = fminf(fmaxf(jf, -1.0f), (float)sh.map_w);
  const float ic = fminf(fmaxf(if_, -1.0f), (float)sh.map_h);
  const int jj = (int)jc, ii = (int)ic;
  const int j0 = min(max(jj, 0), sh.map_w - 1), j1 = min(max(jj + 1, 0), sh.map_w - 1);
  const int i0 = min(max(ii, 0), sh.map_h - 1), i1 = min(max(ii + 1, 0), sh.map_h - 1);
  const float *r0 = map + (size_t)i0 * sh.map_w;
  const float *r1 = map + (size_t)i1 * sh.map_w;
  const float m00 = __ldg(r0 + j0), m01 = __ldg(r0 + j1);
  const float m10 = __ldg(r1 + j0), m11 = __ldg(r1 + j1);
  return (1.0f - a) * (1.0f - b) * m00 + a * (1.0f - b) * m01 + (1.0f - a) * b * m10 + a * b * m11;
}

// The bilinear lookup split in two, so the texel loads can be issued a step before
// they are used: fractional weights (a, b) and the four texels around (p_x, p_y).
__device__ __forceinline__ void tps_costmap_fetch(const TpsShared &sh, const float *map, float px, float py,
                                                  float &a, float &b, float &m00, float &m01, float &m10,
                                                  float &m11) {
  const float fx = (px - sh.origin_x) * sh.inv_res - 0.5f;
  const float fy = (py - sh.origin_y) * sh.inv_res - 0.5f;
  const float jf = floorf(fx), if_ = floorf(fy);
  a = fx - jf;
  b = fy - if_;
  const float jc = fminf(fmaxf(jf, -1.0f), (float)sh.map_w);
  const float ic = fminf(fmaxf(if_, -1.0f), (float)sh.map_h);
  const int jj = (int)jc, ii = (int)ic;
  const int j0 = min(max(jj, 0), sh.map_w - 1), j1 = min(max(jj + 1, 0), sh.map_w - 1);
  const int i0 = min(max(ii, 0), sh.map_h - 1), i1 = min(max(ii + 1, 0), sh.map_h - 1);
  const float *r0 = map + (size_t)i0 * sh.map_w;
  const float *r1 = map + (size_t)i1 * sh.map_w;
  m00 = __ldg(r0 + j0);
  m01 = __ldg(r0 + j1);
  m10 = __ldg(r1 + j0);
  m11 = __ldg(r1 + j1);
}

// State cost at loop index t (Sec. V-C) given the interpolated map value h.
__device__ __forceinline__ float tps_cost_from_h(const TpsShared &sh, float h, float vx, float vy, int t) {
  h = h > sh.map_cap ? sh.map_cap : h;  // NaN stays NaN
  const float zeta = -atan2f(vy, fabsf(vx));
  const float sp = vx - sh.v_des;
  float imp = 0.0f;
  if (h > sh.track_thresh) imp += exp2f((float)t * sh.log2_decay) * sh.crash_cost;
  if (fabsf(zeta) > sh.slip_thresh) imp += sh.crash_cost;
  return sh.w_track * h + sh.w_speed * sp * sp + sh.w_stab * zeta * zeta + sh.w_crash * imp;
}

// State cost at loop index t (Sec. V-C).
__device__ __forceinline__ float tps_state_cost(const TpsShared &sh, const float *map, float px, float py, float vx,
                                                float vy, int t) {
  float h = tps_costmap(sh, map, px, py);
  h = h > sh.map_cap ? sh.map_cap : h;  // NaN stays NaN
  const float zeta = -atan2f(vy, fabsf(vx));
  const float sp = vx - sh.v_des;
  float imp = 0.0f;
  if (h > sh.track_thresh) imp += exp2f((float)t * sh.log2_decay) * sh.crash_cost;
  if (fabsf(zeta) > sh.slip_thresh) imp += sh.crash_cost;
  return sh.w_track * h + sh.w_speed * sp * sp + sh.w_stab * zeta * zeta + sh.w_crash * imp;
}

// The basis-function model (Sec. V-B and the appendix): f = Theta^T phi(x_d, u).  In the
// fast branch tan(alpha) = tan(arctan z) = z, so the slip-angle terms need no arctan / tan.
struct BasisDyn {
  float theta[100];  // [basis i][output o]
  __device__ __forceinline__ void eval(float th, float vx, float vy, float r, float ud, float uF, float &d0,
                                       float &d1, float &d2, float &d3) const {
    float tf, tr, q;
    if (vx > 0.1f) {
      const float iv = 1.0f / vx;
      tf = fmaf(0.45f, r, vy) * iv - ud;
      tr = fmaf(-0.35f, r, vy) * iv;
      q = vy * iv;
    } else {
      tf = -tanf(ud);
      tr = 0.0f;
      q = 0.0f;
    }
    const float sd = sinf(ud);
    const float atf = fabsf(tf), atr = fabsf(tr);
    const float phi[25] = {uF,
                           vx * 0.1f,
                           sd * tf * (1.0f / 1200.0f),
                           sd * tf * atf * (1.0f / 1440000.0f),
                           sd * tf * tf * tf * (1.0f / 1728000000.0f),
                           r * vy * (1.0f / 25.0f),
                           r * 0.1f,
                           vy * 0.1f,
                           sd,
                           q * (1.0f / 40.0f),
                           tf * (1.0f / 1400.0f),
                           tf * atf * (1.0f / 1960000.0f),
                           tf * tf * tf * (1.0f / 2744000000.0f),
                           tr * (1.0f / 40.0f),
                           tr * atr * (1.0f / 1600.0f),
                           tr * tr * tr * (1.0f / 64000.0f),
                           r * vx * (1.0f / 50.0f),
                           th,
                           th * r,
                           th * vx * (1.0f / 3.0f),
                           th * vx * r * (1.0f / 5.0f),
                           vx * vx * 0.01f,
                           vx * vx * vx * 0.001f,
                           uF * uF,
                           uF * uF * uF};
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 25; ++i)
#pragma unroll
      for (int o = 0; o < 4; ++o) d[o] = fmaf(theta[i * 4 + o], phi[i], d[o]);
    d0 = d[0]; d1 = d[1]; d2 = d[2]; d3 = d[3];
  }
};

}  // namespace itmpc
