// iterate_adj.cu -- reverse-mode (adjoint) form of one FP32 IT-MPC iteration for sm_103a.
//
// The paper derives no gradient of its controller; this is the chain rule of
// Alg. 1 (rollout and running cost), Alg. 2 (weights) and the control law of
// Sec. III-D, with the noise held fixed.  Outputs of the iteration are
//   J  = sum_k w_k S_k   and   U'_t = sum_k w_k v_{k,t};
// given cotangents gJ and gU the kernels return d/dtheta [gJ J + sum_t gU_t . U'_t]
// for theta = the four cost multipliers, the nominal sequence and the network.
//
//   adj_scalars_kernel   J, c0 = sum_t gU_t . U'_t and sum of importance weights;
//   adj_backward_kernel  two samples per warp, side by side, so that every W2 element a
//                        lane loads from shared memory feeds both samples' FMAs.  A sample
//                        with w_k = 0 contributes nothing: it runs from the zero state with
//                        a zero cotangent, and a warp whose two samples both have w = 0
//                        skips.  The cost cotangent of sample k is
//                          Sbar_k = w_k (gJ (1 - (S_k - J)/lambda) - (a_k - c0)/lambda),
//                          a_k = sum_t gU_t . v_{k,t}
//                        (dw_k/dS_j = -(1/lambda) w_k (delta_kj - w_j)).  The horizon is
//                        walked backwards in segments of `every` steps: the segment is
//                        re-run forward from its checkpoint x_{t0} (written by the
//                        forward launch), keeping states, controls and both hidden
//                        layers in shared memory; then each step is reversed: cost
//                        slope at x_t, the Euler kinematics, the network (lane j owns
//                        neurons j, j+32, ...; W2 is read from shared memory in both
//                        orientations), the clamp g and the control-cost term.  The
//                        W2 gradient, an outer product summed over samples and steps,
//                        is accumulated by the whole CTA as a small GEMM over the
//                        segment's rows (a2bar x h1) after every segment;
//   adj_reduce_kernel    sums the per-CTA records in a fixed order (deterministic)
//                        and adds the direct term dU'_t/du_t = sum_{importance} w_k.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"

namespace itmpc {

namespace {

constexpr int kAdjWarps = 4;                     // warps per CTA
constexpr int kAdjSPW = 2;                       // samples per warp, side by side
constexpr int kAdjSamples = kAdjWarps * kAdjSPW; // samples per CTA

__host__ __device__ inline int adj_rec_floats(int H, int T) { return (net_floats(H) + 4 + 2 * T + 3) & ~3; }

// Per-sample shared floats for a segment of `every` steps.
__host__ __device__ inline size_t adj_sample_floats(int H, int every) {
  return 8 * (size_t)(every + 1)      // states x_{t0..t0+every}, 8 floats each
         + 4 * (size_t)every          // (v0, v1, g0, g1) per step
         + 4 * (size_t)every          // cost slope (px, py, vx, vy) at x_{t0+1+i}
         + 2 * (size_t)H * every;     // h1 rows, h2 rows (then a2bar rows)
}

__host__ __device__ inline size_t adj_smem_floats(int H, int every, int T) {
  return 2 * (size_t)H * H + kAdjSamples * adj_sample_floats(H, every) + (size_t)kAdjWarps * 2 * T +
         (size_t)adj_rec_floats(H, T);
}

// Slope of the state cost c(x, t) of Sec. V-C with respect to (p_x, p_y, v_x, v_y),
// and the four unweighted terms.  The impulses are piecewise constant (no slope);
// the capped track term has no slope above the cap.
__device__ __forceinline__ void state_cost_slope(const IterParams &p, float px, float py, float vx, float vy, int t,
                                                 float g[4], float comp[4]) {
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
  float h = (1.0f - a) * (1.0f - b) * m00 + a * (1.0f - b) * m01 + (1.0f - a) * b * m10 + a * b * m11;
  g[0] = g[1] = 0.0f;
  if (h > p.map_cap) {
    h = p.map_cap;
  } else {
    g[0] = p.w_track * ((1.0f - b) * (m01 - m00) + b * (m11 - m10)) * p.inv_res;
    g[1] = p.w_track * ((1.0f - a) * (m10 - m00) + a * (m11 - m01)) * p.inv_res;
  }
  const float zeta = -atan2f(vy, fabsf(vx));
  const float sp = vx - p.v_des;
  const float r2 = vx * vx + vy * vy;
  float dzx = 0.0f, dzy = 0.0f;
  if (r2 > 0.0f) {
    const float inv = 1.0f / r2;
    dzx = (vx > 0.0f ? vy : (vx < 0.0f ? -vy : 0.0f)) * inv;
    dzy = -fabsf(vx) * inv;
  }
  g[2] = p.w_speed * 2.0f * sp + p.w_stab * 2.0f * zeta * dzx;
  g[3] = p.w_stab * 2.0f * zeta * dzy;
  float imp = 0.0f;
  if (h > p.track_thresh) imp += exp2f((float)t * p.log2_decay) * p.crash_cost;
  if (fabsf(zeta) > p.slip_thresh) imp += p.crash_cost;
  comp[0] = h;
  comp[1] = sp * sp;
  comp[2] = zeta * zeta;
  comp[3] = imp;
}

// Neumaier compensated running sum.
struct CSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// J = sum_k w_k S_k (w_k != 0), c0 = sum_t gU_t . U'_t, w_imp = sum_{k < n_imp} w_k; one CTA.
__global__ void __launch_bounds__(1024) adj_scalars_kernel(int K, int T, int n_imp, const float *w, const float *S,
                                                           const float *Uo, const float *gUo, const float *gJ,
                                                           float *scal, float *J_out) {
  __shared__ float red[3][32][2];
  CSum j, wi, c;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float wk = w[k];
    if (wk != 0.0f) j.add(wk * S[k]);
    if (k < n_imp) wi.add(wk);
  }
  if (gUo)
    for (int t = threadIdx.x; t < 2 * T; t += blockDim.x) c.add(gUo[t] * Uo[t]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CSum *v[3] = {&j, &c, &wi};
  for (int q = 0; q < 3; ++q) {
    float s = v[q]->s, cc = v[q]->c;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(FULL_MASK, s, o);
      cc += __shfl_xor_sync(FULL_MASK, cc, o);
    }
    if (lane == 0) {
      red[q][warp][0] = s;
      red[q][warp][1] = cc;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float out[3];
    for (int q = 0; q < 3; ++q) {
      CSum t;
      for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) {
        t.add(red[q][i][0]);
        t.add(red[q][i][1]);
      }
      out[q] = t.value();
    }
    scal[0] = out[0];
    scal[1] = out[1];
    scal[2] = out[2];
    scal[3] = gJ ? *gJ : 0.0f;
    if (J_out) *J_out = out[0];
  }
}

template <int H, int ACT>
__global__ void __launch_bounds__(kAdjWarps * 32) adj_backward_kernel(const __grid_constant__ AdjParams a) {
  constexpr int NW = kAdjWarps, SPW = kAdjSPW, SC = kAdjSamples;
  constexpr int M = H / 32;
  constexpr int E = H * H / (NW * 32);  // W2-gradient entries per thread
  constexpr int TJ = 4, TI = E / 4, NIB = H / TI;
  static_assert(E % 4 == 0 && (TI == 2 || TI % 4 == 0), "tile");
  const IterParams &p = a.p;
  const int T = p.T, K = p.K, every = a.every;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t sf = adj_sample_floats(H, every);

  extern __shared__ __align__(16) float sm[];
  float *W2T_s = sm;             // [i][j] = W2[j][i]
  float *W2_s = sm + H * H;      // [j][i] = W2[j][i]
  float *sreg = sm + 2 * H * H;  // SC per-sample regions
  float *ub_s = sreg + SC * sf;  // NW x 2T: per-warp dL/dU of its samples
  float *rec_s = ub_s + NW * 2 * T;
  float *xs[SPW], *vg[SPW], *gc[SPW], *hs1[SPW], *hs2[SPW];
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    xs[q] = sreg + (warp * SPW + q) * sf;
    vg[q] = xs[q] + 8 * (every + 1);
    gc[q] = vg[q] + 4 * every;
    hs1[q] = gc[q] + 4 * every;
    hs2[q] = hs1[q] + H * every;
  }

  const float *net = p.net;
  for (int e = threadIdx.x; e < H * H; e += NW * 32) {
    const float v = __ldg(net + net_off_W2(H) + e);
    W2_s[e] = v;
    W2T_s[(e % H) * H + e / H] = v;
  }
  for (int e = threadIdx.x; e < NW * 2 * T; e += NW * 32) ub_s[e] = 0.0f;
  const int nrec = adj_rec_floats(H, T);
  for (int e = threadIdx.x; e < nrec; e += NW * 32) rec_s[e] = 0.0f;

  float W1r[M][6], b1r[M], b2r[M], W3c[M][4], b3u[4];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = lane + 32 * m;
#pragma unroll
    for (int c = 0; c < 6; ++c) W1r[m][c] = __ldg(net + net_off_W1(H) + j * 6 + c);
    b1r[m] = __ldg(net + net_off_b1(H) + j);
    b2r[m] = __ldg(net + net_off_b2(H) + j);
#pragma unroll
    for (int o = 0; o < 4; ++o) W3c[m][o] = __ldg(net + net_off_W3(H) + o * H + j);
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) b3u[o] = __ldg(net + net_off_b3(H) + o);

  // gradient accumulators: both samples of the warp add into the same registers
  float gW1[M][6], gb1[M], gb2[M], gW3[M][4], gb3[4], gcw[4];
#pragma unroll
  for (int m = 0; m < M; ++m) {
#pragma unroll
    for (int c = 0; c < 6; ++c) gW1[m][c] = 0.0f;
    gb1[m] = gb2[m] = 0.0f;
#pragma unroll
    for (int o = 0; o < 4; ++o) gW3[m][o] = 0.0f;
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) gb3[o] = gcw[o] = 0.0f;
  const int jb = threadIdx.x / NIB, ib = threadIdx.x % NIB;
  float gW2[TJ][TI];
#pragma unroll
  for (int r = 0; r < TJ; ++r)
#pragma unroll
    for (int c = 0; c < TI; ++c) gW2[r][c] = 0.0f;

  // this warp's samples and their cost cotangents; an inactive sample (k >= K or w_k = 0)
  // runs from the zero state with Sbar = 0, so that everything it adds is zero
  int kq[SPW];
  bool act[SPW], impq[SPW];
  float Sbar[SPW];
  const float J = __ldg(a.scal), c0 = __ldg(a.scal + 1), gJ = __ldg(a.scal + 3);
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    const int k = blockIdx.x * SC + warp * SPW + q;
    kq[q] = k;
    impq[q] = k < p.n_imp;
    act[q] = k < K && __ldg(a.w + k) != 0.0f;
    Sbar[q] = 0.0f;
    if (act[q]) {
      float acc = 0.0f;
      if (a.gUo) {
        for (int t = lane; t < T; t += 32) {
          const float2 e = noise_at(p, (uint32_t)k, (uint32_t)t);
          const float v0 = impq[q] ? __ldg(p.U + 2 * t) + e.x : e.x;
          const float v1 = impq[q] ? __ldg(p.U + 2 * t + 1) + e.y : e.y;
          acc = fmaf(__ldg(a.gUo + 2 * t), v0, acc);
          acc = fmaf(__ldg(a.gUo + 2 * t + 1), v1, acc);
        }
        acc = warp_sum(acc);
      }
      Sbar[q] = __ldg(a.w + k) * (gJ * (1.0f - (__ldg(a.S + k) - J) * p.inv_lambda) - (acc - c0) * p.inv_lambda);
    }
  }
  const bool warp_active = act[0] || act[1];
  __syncthreads();

  const float dt = p.dt;
  const int n_ck = T / every + 1;
  const int nseg = (T + every - 1) / every;
  float xb[SPW][7];
#pragma unroll
  for (int q = 0; q < SPW; ++q)
#pragma unroll
    for (int c = 0; c < 7; ++c) xb[q][c] = 0.0f;

  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int t0 = seg * every;
    const int nst = min(every, T - t0);
    if (warp_active) {
      // (a) re-run the segment forward from its checkpoints, both samples side by side
      float x[SPW][7];
#pragma unroll
      for (int q = 0; q < SPW; ++q) {
        const float *ck = a.ckpt + ((size_t)kq[q] * n_ck + seg) * 7;
#pragma unroll
        for (int c = 0; c < 7; ++c) x[q][c] = act[q] ? __ldg(ck + c) : 0.0f;
        if (lane < nst) {
          const int t = t0 + lane;
          const float2 e = noise_at(p, (uint32_t)kq[q], (uint32_t)t);
          const float v0 = impq[q] ? __ldg(p.U + 2 * t) + e.x : e.x;
          const float v1 = impq[q] ? __ldg(p.U + 2 * t + 1) + e.y : e.y;
          *reinterpret_cast<float4 *>(vg[q] + 4 * lane) =
              make_float4(v0, v1, fminf(fmaxf(v0, p.umin0), p.umax0), fminf(fmaxf(v1, p.umin1), p.umax1));
        }
        if (lane < 7) xs[q][lane] = x[q][lane];
      }
      __syncwarp();
      for (int i = 0; i < nst; ++i) {
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          const float z[6] = {x[q][3], x[q][4], x[q][5], x[q][6], vg[q][4 * i + 2], vg[q][4 * i + 3]};
#pragma unroll
          for (int m = 0; m < M; ++m) {
            float acc = b1r[m];
#pragma unroll
            for (int c = 0; c < 6; ++c) acc = fmaf(W1r[m][c], z[c], acc);
            hs1[q][i * H + lane + 32 * m] = activation<ACT>(acc);
          }
        }
        __syncwarp();
        float acc2[SPW][M];
#pragma unroll
        for (int q = 0; q < SPW; ++q)
#pragma unroll
          for (int m = 0; m < M; ++m) acc2[q][m] = b2r[m];
#pragma unroll 4
        for (int ii = 0; ii < H; ii += 4) {
          float4 hv[SPW];
#pragma unroll
          for (int q = 0; q < SPW; ++q) hv[q] = *reinterpret_cast<const float4 *>(hs1[q] + i * H + ii);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float *w = W2T_s + ii * H + lane + 32 * m;
            const float w0 = w[0], w1 = w[H], w2 = w[2 * H], w3 = w[3 * H];
#pragma unroll
            for (int q = 0; q < SPW; ++q) {
              acc2[q][m] = fmaf(w0, hv[q].x, acc2[q][m]);
              acc2[q][m] = fmaf(w1, hv[q].y, acc2[q][m]);
              acc2[q][m] = fmaf(w2, hv[q].z, acc2[q][m]);
              acc2[q][m] = fmaf(w3, hv[q].w, acc2[q][m]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float h2 = activation<ACT>(acc2[q][m]);
            hs2[q][i * H + lane + 32 * m] = h2;
#pragma unroll
            for (int o = 0; o < 4; ++o) d[o] = fmaf(W3c[m][o], h2, d[o]);
          }
#pragma unroll
          for (int o = 0; o < 4; ++o) d[o] = warp_sum(d[o]) + b3u[o];
          float sn, cs;
          sincosf(x[q][2], &sn, &cs);
          const float nx0 = x[q][0] + (cs * x[q][4] - sn * x[q][5]) * dt;
          const float nx1 = x[q][1] + (sn * x[q][4] + cs * x[q][5]) * dt;
          const float nx2 = x[q][2] + x[q][6] * dt;
          x[q][0] = nx0;
          x[q][1] = nx1;
          x[q][2] = nx2;
#pragma unroll
          for (int c = 0; c < 4; ++c) x[q][3 + c] = x[q][3 + c] + d[c] * dt;
          if (lane < 7) xs[q][8 * (i + 1) + lane] = x[q][lane];
        }
      }
      __syncwarp();
      // (b) cost slopes at x_{t0+1 .. t0+nst}, one step per lane; Sbar-weighted components
      if (lane < nst) {
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          const float *xt = xs[q] + 8 * (lane + 1);
          float g4[4], c4[4];
          state_cost_slope(p, xt[0], xt[1], xt[4], xt[5], t0 + lane + 1, g4, c4);
          *reinterpret_cast<float4 *>(gc[q] + 4 * lane) = make_float4(g4[0], g4[1], g4[2], g4[3]);
#pragma unroll
          for (int o = 0; o < 4; ++o) gcw[o] = fmaf(Sbar[q], c4[o], gcw[o]);
        }
      }
      __syncwarp();
      // (c) reverse the segment's steps
      for (int i = nst - 1; i >= 0; --i) {
        const int t = t0 + i;  // step t -> t + 1 used v_t
        float xbp[SPW][7], db[SPW][4];
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          const float4 gci = *reinterpret_cast<const float4 *>(gc[q] + 4 * i);
          xb[q][0] = fmaf(Sbar[q], gci.x, xb[q][0]);
          xb[q][1] = fmaf(Sbar[q], gci.y, xb[q][1]);
          xb[q][4] = fmaf(Sbar[q], gci.z, xb[q][4]);
          xb[q][5] = fmaf(Sbar[q], gci.w, xb[q][5]);
          const float *xp = xs[q] + 8 * i;
          const float th = xp[2], vx = xp[4], vy = xp[5];
          float sn, cs;
          sincosf(th, &sn, &cs);
#pragma unroll
          for (int c = 0; c < 7; ++c) xbp[q][c] = xb[q][c];
          xbp[q][2] += dt * (xb[q][0] * (-sn * vx - cs * vy) + xb[q][1] * (cs * vx - sn * vy));
          xbp[q][4] += dt * (xb[q][0] * cs + xb[q][1] * sn);
          xbp[q][5] += dt * (-xb[q][0] * sn + xb[q][1] * cs);
          xbp[q][6] += dt * xb[q][2];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            db[q][o] = dt * xb[q][3 + o];
            gb3[o] += db[q][o];
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float h2 = hs2[q][i * H + lane + 32 * m];
            float hb = 0.0f;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              hb = fmaf(W3c[m][o], db[q][o], hb);
              gW3[m][o] = fmaf(db[q][o], h2, gW3[m][o]);
            }
            const float a2b = ACT == 1 ? hb : hb * (1.0f - h2 * h2);
            gb2[m] += a2b;
            hs2[q][i * H + lane + 32 * m] = a2b;
          }
        }
        __syncwarp();
        float h1b[SPW][M];
#pragma unroll
        for (int q = 0; q < SPW; ++q)
#pragma unroll
          for (int m = 0; m < M; ++m) h1b[q][m] = 0.0f;
#pragma unroll 4
        for (int jj = 0; jj < H; jj += 4) {
          float4 av[SPW];
#pragma unroll
          for (int q = 0; q < SPW; ++q) av[q] = *reinterpret_cast<const float4 *>(hs2[q] + i * H + jj);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float *w = W2_s + jj * H + lane + 32 * m;
            const float w0 = w[0], w1 = w[H], w2 = w[2 * H], w3 = w[3 * H];
#pragma unroll
            for (int q = 0; q < SPW; ++q) {
              h1b[q][m] = fmaf(w0, av[q].x, h1b[q][m]);
              h1b[q][m] = fmaf(w1, av[q].y, h1b[q][m]);
              h1b[q][m] = fmaf(w2, av[q].z, h1b[q][m]);
              h1b[q][m] = fmaf(w3, av[q].w, h1b[q][m]);
            }
          }
        }
        float ub[2] = {0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          const float *xp = xs[q] + 8 * i;
          const float4 vgi = *reinterpret_cast<const float4 *>(vg[q] + 4 * i);
          const float z[6] = {xp[3], xp[4], xp[5], xp[6], vgi.z, vgi.w};
          float zb[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float h1 = hs1[q][i * H + lane + 32 * m];
            const float a1b = ACT == 1 ? h1b[q][m] : h1b[q][m] * (1.0f - h1 * h1);
            gb1[m] += a1b;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              gW1[m][c] = fmaf(a1b, z[c], gW1[m][c]);
              zb[c] = fmaf(W1r[m][c], a1b, zb[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < 6; ++c) zb[c] = warp_sum(zb[c]);
#pragma unroll
          for (int c = 0; c < 4; ++c) xbp[q][3 + c] += zb[c];
          // the clamp g passes the slope inside [u_min, u_max]; the control-cost term
          // gamma u' Sigma^-1 v adds gamma u/sigma^2 to dL/dv and gamma v/sigma^2 to dL/du
          float vb0 = (vgi.x >= p.umin0 && vgi.x <= p.umax0) ? zb[4] : 0.0f;
          float vb1 = (vgi.y >= p.umin1 && vgi.y <= p.umax1) ? zb[5] : 0.0f;
          float ub0 = 0.0f, ub1 = 0.0f;
          if (p.gamma != 0.0f) {
            const float u0 = __ldg(p.U + 2 * t), u1 = __ldg(p.U + 2 * t + 1);
            const float sg = Sbar[q] * p.gamma;
            vb0 = fmaf(sg * u0, p.inv_sig2_0, vb0);
            vb1 = fmaf(sg * u1, p.inv_sig2_1, vb1);
            ub0 = sg * vgi.x * p.inv_sig2_0;
            ub1 = sg * vgi.y * p.inv_sig2_1;
          }
          if (impq[q]) {
            ub0 += vb0;
            ub1 += vb1;
          }
          ub[0] += ub0;
          ub[1] += ub1;
#pragma unroll
          for (int c = 0; c < 7; ++c) xb[q][c] = xbp[q][c];
        }
        if (lane == 0) {
          ub_s[warp * 2 * T + 2 * t] = ub[0];
          ub_s[warp * 2 * T + 2 * t + 1] = ub[1];
        }
      }
    }
    __syncthreads();
    // (d) W2 gradient: sum over this CTA's active samples and the segment's steps of a2bar h1^T
    for (int sidx = 0; sidx < SC; ++sidx) {
      const int ks = blockIdx.x * SC + sidx;
      if (ks >= K || __ldg(a.w + ks) == 0.0f) continue;
      const float *h1w = sreg + sidx * sf + 8 * (every + 1) + 8 * every;
      const float *a2w = h1w + H * every;
      for (int i = 0; i < nst; ++i) {
        const float4 av = *reinterpret_cast<const float4 *>(a2w + i * H + TJ * jb);
        const float ar[4] = {av.x, av.y, av.z, av.w};
        float hr[TI];
        if constexpr (TI == 2) {
          const float2 hv = *reinterpret_cast<const float2 *>(h1w + i * H + TI * ib);
          hr[0] = hv.x; hr[1] = hv.y;
        } else {
#pragma unroll
          for (int c4 = 0; c4 < TI; c4 += 4) {
            const float4 hv = *reinterpret_cast<const float4 *>(h1w + i * H + TI * ib + c4);
            hr[c4] = hv.x; hr[c4 + 1] = hv.y; hr[c4 + 2] = hv.z; hr[c4 + 3] = hv.w;
          }
        }
#pragma unroll
        for (int r = 0; r < TJ; ++r)
#pragma unroll
          for (int c = 0; c < TI; ++c) gW2[r][c] = fmaf(ar[r], hr[c], gW2[r][c]);
      }
    }
    __syncthreads();
  }

  // ---- this CTA's record: per-warp accumulators summed in warp order ----
  const int nf = net_floats(H);
  for (int w = 0; w < NW; ++w) {
    if (warp == w) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j = lane + 32 * m;
#pragma unroll
        for (int c = 0; c < 6; ++c) rec_s[net_off_W1(H) + j * 6 + c] += gW1[m][c];
        rec_s[net_off_b1(H) + j] += gb1[m];
        rec_s[net_off_b2(H) + j] += gb2[m];
#pragma unroll
        for (int o = 0; o < 4; ++o) rec_s[net_off_W3(H) + o * H + j] += gW3[m][o];
      }
      if (lane == 0) {
#pragma unroll
        for (int o = 0; o < 4; ++o) rec_s[net_off_b3(H) + o] += gb3[o];
      }
      // cost multipliers: the Sbar-weighted components, summed over the lanes' steps
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float c = warp_sum(gcw[o]);
        if (lane == 0) rec_s[nf + o] += c;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < TJ; ++r)
#pragma unroll
    for (int c = 0; c < TI; ++c) rec_s[net_off_W2(H) + (TJ * jb + r) * H + TI * ib + c] = gW2[r][c];
  for (int e = threadIdx.x; e < 2 * T; e += NW * 32) {
    float sum = 0.0f;
    for (int w = 0; w < NW; ++w) sum += ub_s[w * 2 * T + e];
    rec_s[nf + 4 + e] = sum;
  }
  __syncthreads();
  float *rec = a.part + (size_t)blockIdx.x * nrec;
  for (int e = threadIdx.x; e < nrec; e += NW * 32) rec[e] = rec_s[e];
}

// Sum the per-CTA records in CTA order; warp w of a block takes records w, w + 8, ...
// for 32 consecutive outputs, then the 8 partial sums are added in warp order.
__global__ void __launch_bounds__(256) adj_reduce_kernel(int n_cta, int nrec, int nf, int T, const float *part,
                                                         const float *gUo, const float *scal, float *g_net,
                                                         float *g_cw, float *g_U) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const int n_out = nf + 4 + 2 * T;
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
  if (e < n_out) {
    int c = warp;
    for (; c + 24 < n_cta; c += 32) {
      s0 += part[(size_t)c * nrec + e];
      s1 += part[(size_t)(c + 8) * nrec + e];
      s2 += part[(size_t)(c + 16) * nrec + e];
      s3 += part[(size_t)(c + 24) * nrec + e];
    }
    for (; c < n_cta; c += 8) s0 += part[(size_t)c * nrec + e];
  }
  red[warp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (warp == 0 && e < n_out) {
    float s = 0.0f;
    for (int w = 0; w < 8; ++w) s += red[w][lane];
    if (e < nf) {
      g_net[e] = s;
    } else if (e < nf + 4) {
      g_cw[e - nf] = s;
    } else {
      const int t = e - nf - 4;
      g_U[t] = gUo ? fmaf(__ldg(gUo + t), __ldg(scal + 2), s) : s;
    }
  }
}

template <int H, int ACT>
cudaError_t launch_bwd(const AdjParams &a, int n_cta, size_t smem, cudaStream_t s) {
  auto kern = adj_backward_kernel<H, ACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_cta, kAdjWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int adj_num_ctas(int K) { return (K + kAdjSamples - 1) / kAdjSamples; }
size_t adj_part_floats(int K, int H, int T_max) { return (size_t)adj_num_ctas(K) * adj_rec_floats(H, T_max); }
size_t adj_smem_bytes(int H, int every, int T) { return sizeof(float) * adj_smem_floats(H, every, T); }

cudaError_t adj_launch_scalars(int K, int T, int n_imp, const float *w, const float *S, const float *Uo,
                               const float *gUo, const float *gJ, float *scal, float *J_out, cudaStream_t s) {
  adj_scalars_kernel<<<1, 1024, 0, s>>>(K, T, n_imp, w, S, Uo, gUo, gJ, scal, J_out);
  return cudaGetLastError();
}

cudaError_t adj_launch_backward(const AdjParams &a, float *g_cost_w, float *g_U, float *g_net, cudaStream_t s) {
  const int H = a.p.H, T = a.p.T;
  const int n_cta = adj_num_ctas(a.p.K);
  const size_t smem = adj_smem_bytes(H, a.every, T);
  cudaError_t e;
  if (H == 32) e = a.p.activation == 1 ? launch_bwd<32, 1>(a, n_cta, smem, s) : launch_bwd<32, 0>(a, n_cta, smem, s);
  else if (H == 64) e = a.p.activation == 1 ? launch_bwd<64, 1>(a, n_cta, smem, s) : launch_bwd<64, 0>(a, n_cta, smem, s);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  const int nf = net_floats(H);
  const int n_out = nf + 4 + 2 * T;
  adj_reduce_kernel<<<(n_out + 31) / 32, 256, 0, s>>>(n_cta, adj_rec_floats(H, T), nf, T, a.part, a.gUo, a.scal,
                                                      g_net, g_cost_w, g_U);
  return cudaGetLastError();
}

}  // namespace itmpc
