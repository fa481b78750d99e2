// iterate_h32.cu -- the fused FP32 IT-MPC iteration for the paper's 6 -> 32 -> 32 -> 4
// network (Sec. V-B) on sm_103a: noise, rollout, running cost, weights and update of
// Alg. 1 / Alg. 2 in one launch.
//
// A warp owns one sample and lane j owns hidden neuron j of both layers; a CTA owns
// NW consecutive samples.  Per step the only serial work is the network:
//   Layers 3 and 1 are affine, so with M = dt W1x W3 (32 x 32), beta = dt W1x b3 and
//   the Euler step x_d(t+1) = x_d(t) + dt d(t), d(t) = W3 h2(t) + b3, the layer-1
//   pre-activation obeys
//     a1(t+1) = a1(t) + M h2(t) + beta + W1u (g(t+1) - g(t))
//   (W1x, W1u the state and control columns of W1, g the clamped control).  A step is
//   then two 32-term dot products, each behind a tanh: h1 = tanh(a1) is broadcast
//   through a shared row, h2 = tanh(W2 h1 + b2) through a 32-row ring, and the lane's
//   rows of W2 and M are packed FP32 pairs in registers, multiplied two terms per
//   instruction (fma.rn.f32x2) against 16-byte shared loads.  a1 is carried as a
//   compensated (Kahan) sum.
// Everything else is done every 32 steps, with lane = step, by the same warp (block
// epilogue): the output layer d = W3 h2 + b3 from the ring, x_d, heading and position
// by warp prefix sums (explicit Euler from the old state), the running cost of
// Sec. V-C at x(t+1) plus the control-cost term of Sec. III-E, and the noise of the
// block after next.  The four costmap texels of a step are loaded one block before
// they are used, so the fetch latency hides behind 32 steps of the recurrence.
// The CTA's partial record and the merge are those of the other fused kernel
// (itmpc_fused.cuh).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_fused.cuh"
#include "itmpc_merge.cuh"
#include "itmpc_sum.cuh"

namespace itmpc {

namespace {

constexpr int kH = 32;
constexpr int kRingStride = 36;  // padded ring row: lanes reading rows t, t + 1, ... hit distinct banks

__host__ __device__ constexpr size_t al16(size_t n) { return (n + 15) & ~size_t(15); }

// Shared memory of a CTA of nw warps for horizon T: U, W3 | b3, S and e of the CTA's
// samples, then one block per warp [h1 row | h2 ring | g(v) over t | eps over t].
struct H32Layout {
  size_t U, W3b3, S, e, warps, per_warp, hrow, ring, gv, eps, total;
};

__host__ __device__ inline H32Layout h32_layout(int T, int nw) {
  H32Layout L{};
  size_t off = 0;
  L.U = off;    off += al16(sizeof(float) * 2 * (size_t)T);
  L.W3b3 = off; off += al16(sizeof(float) * (4 * kH + 4));
  L.S = off;    off += al16(sizeof(float) * (size_t)nw);
  L.e = off;    off += al16(sizeof(float) * (size_t)nw);
  L.hrow = 0;
  L.ring = L.hrow + al16(sizeof(float) * kH);
  L.gv = L.ring + al16(sizeof(float) * 32 * kRingStride);
  L.eps = L.gv + al16(sizeof(float2) * (size_t)T);
  L.per_warp = L.eps + al16(sizeof(float2) * (size_t)T);
  L.warps = off; off += L.per_warp * (size_t)nw;
  L.total = off;
  return L;
}

typedef unsigned long long u64;

// (x.lo + x.hi) + (y.lo + y.hi) of two packed partial-sum pairs
__device__ __forceinline__ float pair_total(u64 x, u64 y) {
  const float2 a = f2unpack(x), b = f2unpack(y);
  return (a.x + a.y) + (b.x + b.y);
}

// Noise of steps t0 .. t0 + 31 of sample k (lane = step): eps and g(v) into the warp's rows.
__device__ __forceinline__ void noise_block(const IterParams &p, int k, bool imp, uint32_t c2, uint32_t c3, int t0,
                                            const float *U_s, float2 *gv, float2 *eps, int lane) {
  const int t = t0 + lane;
  if (t >= p.T) return;
  const uint4 w = philox4x32_10(make_uint4(p.k_base + (uint32_t)k, (uint32_t)t, c2, c3), p.key0, p.key1);
  const float2 z = box_muller(w.x, w.y);
  const float2 e = make_float2(p.sigma0 * z.x, p.sigma1 * z.y);
  if (p.eps_out) reinterpret_cast<float2 *>(p.eps_out)[(size_t)k * p.T + t] = e;
  const float v0 = imp ? U_s[2 * t] + e.x : e.x;
  const float v1 = imp ? U_s[2 * t + 1] + e.y : e.y;
  eps[t] = e;
  gv[t] = make_float2(fminf(fmaxf(v0, p.umin0), p.umax0), fminf(fmaxf(v1, p.umin1), p.umax1));
}

// A step's costmap lookup split in two: the texels are loaded in one block epilogue
// and combined in the next.
struct PendingCost {
  float a, b, m00, m01, m10, m11, vx, vy;
  int t;  // loop index of the cost (1..T); 0: nothing pending
};

__device__ __forceinline__ void cost_fetch(const IterParams &p, float px, float py, PendingCost &c) {
  const float fx = (px - p.origin_x) * p.inv_res - 0.5f;
  const float fy = (py - p.origin_y) * p.inv_res - 0.5f;
  const float jf = floorf(fx), if_ = floorf(fy);
  c.a = fx - jf;
  c.b = fy - if_;
  const float jc = fminf(fmaxf(jf, -1.0f), (float)p.map_w);
  const float ic = fminf(fmaxf(if_, -1.0f), (float)p.map_h);
  const int jj = (int)jc, ii = (int)ic;  // NaN positions give index 0: still in range
  const int j0 = min(max(jj, 0), p.map_w - 1), j1 = min(max(jj + 1, 0), p.map_w - 1);
  const int i0 = min(max(ii, 0), p.map_h - 1), i1 = min(max(ii + 1, 0), p.map_h - 1);
  const float *r0 = p.map + (size_t)i0 * p.map_w;
  const float *r1 = p.map + (size_t)i1 * p.map_w;
  c.m00 = __ldg(r0 + j0);
  c.m01 = __ldg(r0 + j1);
  c.m10 = __ldg(r1 + j0);
  c.m11 = __ldg(r1 + j1);
}

// State cost of Sec. V-C at loop index c.t from the fetched texels (NaN positions give NaN).
__device__ __forceinline__ float cost_finish(const IterParams &p, const PendingCost &c) {
  const float a = c.a, b = c.b;
  float h = (1.0f - a) * (1.0f - b) * c.m00 + a * (1.0f - b) * c.m01 + (1.0f - a) * b * c.m10 + a * b * c.m11;
  h = h > p.map_cap ? p.map_cap : h;  // NaN stays NaN
  const float zeta = -atan2f(c.vy, fabsf(c.vx));
  const float sp = c.vx - p.v_des;
  float imp = 0.0f;
  if (h > p.track_thresh) imp += exp2f((float)c.t * p.log2_decay) * p.crash_cost;
  if (fabsf(zeta) > p.slip_thresh) imp += p.crash_cost;
  return p.w_track * h + p.w_speed * sp * sp + p.w_stab * zeta * zeta + p.w_crash * imp;
}

template <int NW, int ACT>
__global__ void __launch_bounds__(NW * 32, 1) iterate_h32_kernel(const __grid_constant__ IterParams p) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = p.T;
  const H32Layout L = h32_layout(T, NW);
  float *U_s = reinterpret_cast<float *>(smem + L.U);
  float *W3b3_s = reinterpret_cast<float *>(smem + L.W3b3);
  float *S_s = reinterpret_cast<float *>(smem + L.S);
  float *e_s = reinterpret_cast<float *>(smem + L.e);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char *wblk = smem + L.warps + L.per_warp * warp;
  float *hrow = reinterpret_cast<float *>(wblk + L.hrow);
  float *ring = reinterpret_cast<float *>(wblk + L.ring);
  float2 *gv = reinterpret_cast<float2 *>(wblk + L.gv);
  float2 *eps = reinterpret_cast<float2 *>(wblk + L.eps);
  const int k0 = blockIdx.x * NW;
  const int k = k0 + warp;
  const float *net = p.net;

  // ---- prologue: nominal controls, W3 | b3, the map slice into L2, Philox counter words ----
  unsigned gen0 = 0;
  if (p.coop && tid == 0) gen0 = ld_acquire_u32(p.grid_bar + 1);  // generation before this launch's barrier
  if (tid == 0 && (reinterpret_cast<uintptr_t>(p.map) & 15) == 0) {
    // bring this CTA's slice of the costmap into L2 while the rollouts start
    const size_t bytes = sizeof(float) * (size_t)p.map_w * p.map_h;
    const size_t chunk = ((bytes + gridDim.x - 1) / gridDim.x + 15) & ~size_t(15);
    const size_t beg = chunk * blockIdx.x;
    if (beg < bytes) {
      const size_t n = ((bytes - beg < chunk ? bytes - beg : chunk)) & ~size_t(15);
      for (size_t off = 0; off < n; off += 65536) {
        const uint32_t sz = (uint32_t)(n - off < 65536 ? n - off : 65536);
        prefetch_l2(reinterpret_cast<const char *>(p.map) + beg + off, sz);
      }
    }
  }
  for (int i = tid; i < 2 * T; i += NT) U_s[i] = __ldg(p.U + i);
  for (int i = tid; i < 4 * kH + 4; i += NT) W3b3_s[i] = __ldg(net + net_off_W3(kH) + i);  // W3 then b3
  uint32_t c2 = p.ctr2, c3 = p.ctr3;
  if (p.iter_add != nullptr) {  // a replayed graph's device-side offset of the iteration index
    const unsigned long long it = (((unsigned long long)(c3 & 0xFFFFu) << 32) | c2) + *p.iter_add;
    c2 = (uint32_t)it;
    c3 = (c3 & 0xFFFF0000u) | (uint32_t)((it >> 32) & 0xFFFFu);
  }
  __syncthreads();

  float S_total = 0.0f;
  if (k < p.K) {  // warp-uniform
    const bool imp = (long long)p.k_base + k < p.n_imp;  // the exploration split counts global samples
    const float dt = p.dt;
    const int j = lane;
    // the lane's network slice: W1 row j, b1, b2, its W2 row and M row as packed pairs
    float w1x[4], b3[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      w1x[o] = __ldg(net + net_off_W1(kH) + j * 6 + o);
      b3[o] = W3b3_s[4 * kH + o];
    }
    const float w1u0 = __ldg(net + net_off_W1(kH) + j * 6 + 4), w1u1 = __ldg(net + net_off_W1(kH) + j * 6 + 5);
    const float b2 = __ldg(net + net_off_b2(kH) + j);
    float beta = 0.f;
#pragma unroll
    for (int o = 0; o < 4; ++o) beta = fmaf(dt * w1x[o], b3[o], beta);
    u64 w2[16], mr[16];
    {
      const float *w2row = net + net_off_W2(kH) + j * kH;
#pragma unroll
      for (int i = 0; i < kH; i += 2) w2[i / 2] = f2pack(__ldg(w2row + i), __ldg(w2row + i + 1));
#pragma unroll
      for (int i = 0; i < kH; i += 2) {
        float m0 = 0.f, m1 = 0.f;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          m0 = fmaf(w1x[o], W3b3_s[o * kH + i], m0);
          m1 = fmaf(w1x[o], W3b3_s[o * kH + i + 1], m1);
        }
        mr[i / 2] = f2pack(dt * m0, dt * m1);
      }
    }
    // noise of the first two blocks (the epilogue of block b draws block b + 2)
    noise_block(p, k, imp, c2, c3, 0, U_s, gv, eps, lane);
    noise_block(p, k, imp, c2, c3, 32, U_s, gv, eps, lane);
    __syncwarp();
    // a1(0) = b1 + W1x x_d(0) + W1u g(0)
    float2 g = gv[0];
    float a1 = __ldg(net + net_off_b1(kH) + j);
#pragma unroll
    for (int o = 0; o < 4; ++o) a1 = fmaf(w1x[o], __ldg(p.x0 + 3 + o), a1);
    a1 = fmaf(w1u0, g.x, fmaf(w1u1, g.y, a1));
    float comp = 0.f;  // Kahan compensation of a1

    // carries of the block epilogues (every lane holds the same values): x_d(t0), theta, p
    float4 xd_c = make_float4(__ldg(p.x0 + 3), __ldg(p.x0 + 4), __ldg(p.x0 + 5), __ldg(p.x0 + 6));
    float th_c = __ldg(p.x0 + 2), px_c = __ldg(p.x0 + 0), py_c = __ldg(p.x0 + 1);
    const int every = p.states_every > 0 ? p.states_every : 1;
    const bool dbg = p.states_out != nullptr && k < p.n_states;
    float *st_o = dbg ? p.states_out + (size_t)k * (T / every + 1) * 7 : nullptr;
    if (dbg && lane < 7) st_o[lane] = __ldg(p.x0 + lane);
    PendingCost pend;
    pend.t = 0;
    CSum S;  // this lane's share of S_k = sum_t c_t (steps t = lane mod 32), compensated
    const ulonglong2 *hrow2 = reinterpret_cast<const ulonglong2 *>(hrow);
    const ulonglong2 *W3p = reinterpret_cast<const ulonglong2 *>(W3b3_s);

    for (int t = 0; t < T; ++t) {
      // layer 2: h2 = tanh(W2 tanh(a1) + b2)
      hrow[j] = activation<ACT>(a1);
      __syncwarp();
      u64 acc0 = f2pack(b2, 0.f), acc1 = 0ull;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const ulonglong2 hv = hrow2[m];
        acc0 = ffma2(w2[2 * m], hv.x, acc0);
        acc1 = ffma2(w2[2 * m + 1], hv.y, acc1);
      }
      float *row = ring + (t & 31) * kRingStride;
      row[j] = activation<ACT>(pair_total(acc0, acc1));
      __syncwarp();
      // a1(t + 1) = a1(t) + M h2(t) + beta + W1u (g(t + 1) - g(t))
      if (t + 1 < T) {
        const float2 gn = gv[t + 1];
        const ulonglong2 *row2 = reinterpret_cast<const ulonglong2 *>(row);
        u64 e0 = f2pack(fmaf(w1u0, gn.x - g.x, beta), w1u1 * (gn.y - g.y)), e1 = 0ull;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const ulonglong2 hv = row2[m];
          e0 = ffma2(mr[2 * m], hv.x, e0);
          e1 = ffma2(mr[2 * m + 1], hv.y, e1);
        }
        const float y = pair_total(e0, e1) - comp;
        const float s = a1 + y;
        comp = (s - a1) - y;
        a1 = s;
        g = gn;
      }
      if ((t & 31) != 31 && t + 1 != T) continue;

      // ---- block epilogue: steps t0 .. t, lane = step ----
      const int t0 = t & ~31;
      const int ts = t0 + lane;
      const bool valid = ts <= t;
      // d(ts) = W3 h2(ts) + b3 from the ring row of step ts
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) {
        const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(ring + lane * kRingStride);
        u64 q[4][2];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          q[o][0] = f2pack(b3[o], 0.f);
          q[o][1] = 0ull;
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const ulonglong2 hv = r2[m];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const ulonglong2 wv = W3p[o * 8 + m];
            q[o][0] = ffma2(wv.x, hv.x, q[o][0]);
            q[o][1] = ffma2(wv.y, hv.y, q[o][1]);
          }
        }
        d = make_float4(pair_total(q[0][0], q[0][1]), pair_total(q[1][0], q[1][1]), pair_total(q[2][0], q[2][1]),
                        pair_total(q[3][0], q[3][1]));
      }
      // x_d(ts + 1) = x_d(t0) + dt sum_{s <= ts} d(s); x_d(ts) the exclusive sum
      const float i0 = warp_incl_scan(dt * d.x, lane), i1 = warp_incl_scan(dt * d.y, lane);
      const float i2 = warp_incl_scan(dt * d.z, lane), i3 = warp_incl_scan(dt * d.w, lane);
      float e0 = __shfl_up_sync(FULL_MASK, i0, 1), e1 = __shfl_up_sync(FULL_MASK, i1, 1);
      float e2 = __shfl_up_sync(FULL_MASK, i2, 1), e3 = __shfl_up_sync(FULL_MASK, i3, 1);
      if (lane == 0) e0 = e1 = e2 = e3 = 0.f;
      float4 xo = make_float4(xd_c.x + e0, xd_c.y + e1, xd_c.z + e2, xd_c.w + e3);  // x_d(ts)
      const float4 xn = make_float4(xd_c.x + i0, xd_c.y + i1, xd_c.z + i2, xd_c.w + i3);  // x_d(ts + 1)
      xd_c.x += __shfl_sync(FULL_MASK, i0, 31);
      xd_c.y += __shfl_sync(FULL_MASK, i1, 31);
      xd_c.z += __shfl_sync(FULL_MASK, i2, 31);
      xd_c.w += __shfl_sync(FULL_MASK, i3, 31);
      if (!valid) xo = make_float4(0.f, 0.f, 0.f, 0.f);
      // heading and position: explicit Euler from the old state (Sec. V-B)
      const float incl_th = warp_incl_scan(dt * xo.w, lane);
      float excl_th = __shfl_up_sync(FULL_MASK, incl_th, 1);
      if (lane == 0) excl_th = 0.0f;
      float sn, cs;
      sincosf(th_c + excl_th, &sn, &cs);
      const float incl_px = warp_incl_scan(dt * (cs * xo.y - sn * xo.z), lane);
      const float incl_py = warp_incl_scan(dt * (sn * xo.y + cs * xo.z), lane);
      const float pxn = px_c + incl_px, pyn = py_c + incl_py, thn = th_c + incl_th;  // x(ts + 1)
      th_c += __shfl_sync(FULL_MASK, incl_th, 31);
      px_c += __shfl_sync(FULL_MASK, incl_px, 31);
      py_c += __shfl_sync(FULL_MASK, incl_py, 31);
      // the previous block's running costs (texels loaded one block ago), then this block's fetch
      if (pend.t > 0) S.add(cost_finish(p, pend));
      pend.t = 0;
      if (valid) {
        cost_fetch(p, pxn, pyn, pend);
        pend.vx = xn.y;
        pend.vy = xn.z;
        pend.t = ts + 1;
        if (p.gamma != 0.0f) {  // gamma u_{t}' Sigma^-1 v_{t} with the unclamped v (Sec. III-E)
          const float2 e = eps[ts];
          const float u0 = U_s[2 * ts], u1 = U_s[2 * ts + 1];
          const float v0 = imp ? u0 + e.x : e.x, v1 = imp ? u1 + e.y : e.y;
          S.add(p.gamma * (u0 * v0 * p.inv_sig2_0 + u1 * v1 * p.inv_sig2_1));
        }
        if (dbg && (ts + 1) % every == 0) {
          float *o = st_o + (size_t)((ts + 1) / every) * 7;
          o[0] = pxn; o[1] = pyn; o[2] = thn; o[3] = xn.x; o[4] = xn.y; o[5] = xn.z; o[6] = xn.w;
        }
      }
      if (t0 + 64 < T) noise_block(p, k, imp, c2, c3, t0 + 64, U_s, gv, eps, lane);
      __syncwarp();  // the ring and the noise rows are consistent for the next block
    }
    if (pend.t > 0) S.add(cost_finish(p, pend));
    S_total = csum_warp(S).value();
    if (lane == 0) p.costs[k] = S_total;
  } else {
    // a sample past K: its weight is 0, and its noise row must hold numbers for the E sums
    for (int t = lane; t < T; t += 32) eps[t] = make_float2(0.0f, 0.0f);
  }
  if (lane == 0) S_s[warp] = S_total;
  __syncthreads();

  // ---- the CTA's partial record and the merge (itmpc_fused.cuh) ----
  record_and_merge<NT, NW>(p, S_s, e_s, reinterpret_cast<const float *>(smem + L.warps + L.eps), L.per_warp / 4,
                           k0, gen0, reinterpret_cast<float *>(smem + L.warps));
}

constexpr int kWarpChoices[] = {1, 2, 4, 7, 8, 12, 14, 16};

template <int NW, int ACT>
cudaError_t launch_nw(const IterParams &p, int group, cudaStream_t s) {
  const H32Layout L = h32_layout(p.T, NW);
  auto kern = iterate_h32_kernel<NW, ACT>;
  DeviceInfo di;
  cudaError_t e = device_info(di);
  if (e != cudaSuccess) return e;
  const int nC = (p.K + NW - 1) / NW;
  // Shared memory for staging one merge (all of a group's records) when the
  // occupancy the grid needs still fits; otherwise the merge works in chunks.
  const int per_merge = nC <= group ? nC : group;
  const size_t PLb = sizeof(float) * (size_t)partial_len(p.T);
  const size_t want = L.warps + sizeof(float) * (size_t)((per_merge + 3) & ~3) + PLb * per_merge;
  const int ctas_per_sm = (nC + di.sms - 1) / di.sms;
  size_t budget = di.smem_per_sm / (size_t)ctas_per_sm;
  budget = budget > 1024 ? budget - 1024 : 0;  // per-CTA reservation
  if (budget > di.smem_optin) budget = di.smem_optin;
  size_t smem = L.total;
  if (want > smem && want <= budget) smem = want;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  static size_t configured[64] = {};  // largest dynamic shared memory size set so far, per device
  if (smem > configured[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = smem;
  }
  IterParams q = p;
  q.group = group;
  q.stage_floats = (int)((smem - L.warps) / sizeof(float));
  // Cooperative launch when every CTA can be resident at once and the U' slices fit
  // the tail's per-CTA bound; otherwise the last-CTA merge tree.
  static int occ_per_sm[64] = {};
  static size_t occ_smem[64] = {};
  if (occ_smem[dev] != smem) {
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NW * 32, smem)) != cudaSuccess) return e;
    occ_per_sm[dev] = per;
    occ_smem[dev] = smem;
  }
  const int per_sm = occ_per_sm[dev];
  const int T2 = 2 * p.T;
  q.coop = (per_sm * di.sms >= nC) && (nC <= 2 * NW * 32) && ((T2 + nC - 1) / nC <= 8) && p.grid_bar != nullptr &&
           p.rec_out == nullptr;  // a shard's merged record comes from the merge tree
  if (q.coop) {
    void *args[] = {(void *)&q};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(nC), dim3(NW * 32), args, smem, s);
    if (e == cudaSuccess) return cudaSuccess;
    cudaGetLastError();  // fall back to the ordinary launch
    q.coop = 0;
  }
  kern<<<nC, NW * 32, smem, s>>>(q);
  return cudaGetLastError();
}

}  // namespace

int h32_pick_warps(int K, int T, size_t smem_limit) {
  DeviceInfo di;
  const int sms = device_info(di) == cudaSuccess && di.sms > 0 ? di.sms : 148;
  // spread the samples evenly over the SMs: the smallest CTA that needs one CTA per SM
  const int want = (K + sms - 1) / sms;
  constexpr int n_choices = (int)(sizeof(kWarpChoices) / sizeof(int));
  int i = n_choices - 1;
  for (int c = 0; c < n_choices; ++c)
    if (kWarpChoices[c] >= want) {
      i = c;
      break;
    }
  // smaller CTAs while the shared memory does not fit, never below min(4, want):
  // the scratch sizes (h32_max_ctas) rely on that floor
  const int floor_nw = want < 4 ? want : 4;
  while (i > 0 && kWarpChoices[i - 1] >= floor_nw && h32_layout(T, kWarpChoices[i]).total > smem_limit) --i;
  return kWarpChoices[i];
}

size_t h32_smem_bytes(int T, int nw) { return h32_layout(T, nw).total; }

size_t h32_max_ctas(int K) {
  DeviceInfo di;
  const size_t sms = device_info(di) == cudaSuccess && di.sms > 0 ? (size_t)di.sms : 160;
  const size_t by4 = ((size_t)K + 3) / 4;
  return by4 > sms ? by4 : sms;
}

cudaError_t h32_launch_iterate(const IterParams &p, int nw, int group, cudaStream_t s) {
#define ITMPC_H32(WW)                                                                       \
  if (nw == WW) return p.activation == 1 ? launch_nw<WW, 1>(p, group, s) : launch_nw<WW, 0>(p, group, s);
  ITMPC_H32(1)
  ITMPC_H32(2)
  ITMPC_H32(4)
  ITMPC_H32(7)
  ITMPC_H32(8)
  ITMPC_H32(12)
  ITMPC_H32(14)
  ITMPC_H32(16)
#undef ITMPC_H32
  return cudaErrorInvalidConfiguration;
}

}  // namespace itmpc
