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
//                        (dw_k/dS_j = -(1/lambda) w_k (delta_kj - w_j)).  One CTA per SM,
//                        its warp count (8-16) spreading K over the SMs.  The horizon is
//                        walked backwards in segments of `every` steps: the segment is re-run
//                        forward from its checkpoint x_{t0} (written by the forward launch),
//                        keeping its states, controls and hidden-layer rows in shared memory
//                        (in sub-segments, each re-run from its stored start state, when the
//                        rows do not fit).  Each step is then reversed: cost slope at x_t, the
//                        Euler kinematics, the network (both matrix-vector products on 4 x 32
//                        register tiles; one copy of W2 with padded rows serves both
//                        orientations without bank conflicts), the clamp g and the
//                        control-cost term.  The W2 gradient, an outer product summed over
//                        samples and steps, is a small GEMM over the segment's rows
//                        (a2bar x h1) by two 128-thread groups, added to the CTA's record
//                        in place;
//   adj_reduce_kernel    sums the per-CTA records in a fixed order (deterministic)
//                        and adds the direct term dU'_t/du_t = sum_{importance} w_k.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"

namespace itmpc {

namespace {

constexpr int kAdjSPW = 2;                       // samples per warp, side by side
constexpr int kAdjMinWarps = 8, kAdjMaxWarps = 16; // warps per CTA: one CTA per SM
constexpr int kAdjDThreads = 128;                // threads per group in the W2-gradient GEMM (two groups)

// Warps per CTA: the samples spread over one CTA per SM (two per warp), 8..16 warps.
inline int adj_warps(int K, int n_sm) {
  const int per_sm = (K + n_sm - 1) / n_sm;
  const int nw = (per_sm + kAdjSPW - 1) / kAdjSPW;
  return nw < kAdjMinWarps ? kAdjMinWarps : (nw > kAdjMaxWarps ? kAdjMaxWarps : nw);
}

__host__ __device__ inline int adj_rec_floats(int H, int T) { return (net_floats(H) + 4 + 2 * T + 3) & ~3; }
// A CTA's slot in the record buffer: its record, then one dL/dU row (2T) per warp.
__host__ __device__ inline size_t adj_cta_floats(int H, int T, int nw) {
  return (size_t)adj_rec_floats(H, T) + (size_t)nw * 2 * T;
}
__host__ __device__ inline int adj_w2_stride(int H) { return H + 4; }

// Per-sample shared floats for a segment of `every` steps walked in sub-segments of `sub`
// steps: states and controls for the whole segment, hidden-layer rows for one sub-segment.
__host__ __device__ inline size_t adj_sample_floats(int H, int every, int sub) {
  return 8 * (size_t)(every + 1)    // states x_{t0..t0+every}, 8 floats each
         + 4 * (size_t)every        // (v0, v1, g0, g1) per step
         + 4 * (size_t)every        // cost slope (px, py, vx, vy) at x_{t0+1+i}
         + 2 * (size_t)H * sub;     // h1 rows, h2 rows (then a2bar rows) of the sub-segment
}

// The per-sample regions; the CTA's record reuses them once the last segment is done.
__host__ __device__ inline size_t adj_region_floats(int H, int every, int sub, int T, int nw) {
  const size_t s = (size_t)kAdjSPW * nw * adj_sample_floats(H, every, sub);
  const size_t r = (size_t)adj_rec_floats(H, T);
  return s > r ? s : r;
}

// W3 by neuron (4 floats each), b1, b2, and 8 per-warp sums (b3 gradient, cost components)
__host__ __device__ inline int adj_small_floats(int H, int nw) { return 6 * H + 8 * nw; }

// W2 (rows padded), the small tables, then the per-sample regions.
__host__ __device__ inline size_t adj_smem_floats(int H, int every, int sub, int T, int nw) {
  return (size_t)H * adj_w2_stride(H) + adj_small_floats(H, nw) + adj_region_floats(H, every, sub, T, nw);
}

// The longest sub-segment (every, every/2, every/3, ...) whose footprint fits a CTA;
// a sub-segment other than the segment's last is re-run from its stored start state.
inline int adj_sub_len(int H, int every, int T, int nw, size_t smem_max) {
  for (int n = 1; n <= every; ++n) {
    const int sub = (every + n - 1) / n;
    if (sizeof(float) * adj_smem_floats(H, every, sub, T, nw) <= smem_max) return sub;
  }
  return 1;
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
__global__ void __launch_bounds__(kAdjMaxWarps * 32, 1) adj_backward_kernel(const __grid_constant__ AdjParams a) {
  constexpr int SPW = kAdjSPW;
  constexpr int M = H / 32;
  constexpr int WS = H + 4;             // padded W2 row: conflict-free in both orientations
  constexpr int NTD = kAdjDThreads;
  constexpr int E = H * H / NTD;         // W2-gradient entries per thread
  constexpr int TJ = E >= 8 ? 4 : 2, TI = E / TJ, NIB = H / TI;
  static_assert(E % 4 == 0 && (TI == 2 || TI % 4 == 0), "tile");
  const IterParams &p = a.p;
  const int T = p.T, K = p.K, every = a.every, sub = a.sub;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NW = blockDim.x >> 5, SC = SPW * NW, NT = blockDim.x;
  const size_t sf = adj_sample_floats(H, every, sub);

  extern __shared__ __align__(16) float sm[];
  float *W2_s = sm;                    // [j][i] = W2[j][i], rows WS floats apart
  float *W3_s = sm + H * WS;           // [j][o] = W3[o][j]
  float *b1_s = W3_s + 4 * H, *b2_s = b1_s + H;
  float *wsum_s = b2_s + H;            // NW x 8: per-warp b3 gradient (4), cost components (4)
  // (b2_s + H and wsum_s + 8 NW are 16-byte aligned: H and 8 NW are multiples of 4)
  float *sreg = wsum_s + 8 * NW;       // SC per-sample regions; the CTA's record at the end
  float *xs[SPW], *vg[SPW], *gc[SPW], *hs1[SPW], *hs2[SPW];
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    xs[q] = sreg + (warp * SPW + q) * sf;
    vg[q] = xs[q] + 8 * (every + 1);
    gc[q] = vg[q] + 4 * every;
    hs1[q] = gc[q] + 4 * every;
    hs2[q] = hs1[q] + H * sub;
  }

  const float *net = p.net;
  for (int e = threadIdx.x; e < H * H; e += NT) W2_s[(e / H) * WS + e % H] = __ldg(net + net_off_W2(H) + e);
  for (int e = threadIdx.x; e < 4 * H; e += NT) W3_s[e] = __ldg(net + net_off_W3(H) + (e & 3) * H + (e >> 2));
  for (int e = threadIdx.x; e < H; e += NT) {
    b1_s[e] = __ldg(net + net_off_b1(H) + e);
    b2_s[e] = __ldg(net + net_off_b2(H) + e);
  }
  for (int e = threadIdx.x; e < 8 * NW; e += NT) wsum_s[e] = 0.0f;
  const int nrec = adj_rec_floats(H, T);
  float *rec = a.part + (size_t)blockIdx.x * adj_cta_floats(H, T, NW);
  float *ub_w = rec + nrec + (size_t)warp * 2 * T;  // this warp's dL/dU row (written while it runs)

  // Register tiles of the two matrix-vector products (H/16 rows or columns per lane, half of
  // the other dimension; one shuffle exchange finishes the sums):
  //   W2 h1:     lane (r4, ch) sums rows r4 + 16 rr over columns [H/2 ch, H/2 ch + H/2) and
  //              keeps rows lane + 32 m (layer-2 neuron j = lane + 32 m);
  //   W2^T a2b:  lane (r4, ch) sums columns CW r4 .. + CW-1 over rows [H/2 ch, ...) and keeps
  //              columns CW r4 + M ch + m (layer-1 neuron i1(m)).
  constexpr int R = H / 16, CW = H / 16, HH = H / 2;
  const int r4 = lane & 15, ch = lane >> 4;
  const int i1 = CW * r4 + M * ch;  // first layer-1 neuron of this lane (i1 + m, m < M)
  float W1r[M][6];
#pragma unroll
  for (int m = 0; m < M; ++m) {
#pragma unroll
    for (int c = 0; c < 6; ++c) W1r[m][c] = __ldg(net + net_off_W1(H) + (i1 + m) * 6 + c);
  }

  // gradient accumulators: both samples of the warp add into the same registers
  float gW1[M][6], gb1[M], gb2[M], gW3[M][4];
#pragma unroll
  for (int m = 0; m < M; ++m) {
#pragma unroll
    for (int c = 0; c < 6; ++c) gW1[m][c] = 0.0f;
    gb1[m] = gb2[m] = 0.0f;
#pragma unroll
    for (int o = 0; o < 4; ++o) gW3[m][o] = 0.0f;
  }
  // this thread's W2-gradient tile: rows TJ*jb .. +3; columns in groups of 4 (TI = 2: one pair),
  // group g at 4*ib + 4*NIB*g, so that a quarter-warp's 16-byte loads are contiguous
  // Two groups of NTD threads (warps 0..7) take half of the CTA's samples each and add into
  // the record in turn; the other warps wait at the barriers.
  const int dhalf = threadIdx.x < 2 * NTD ? threadIdx.x / NTD : 2, dtid = threadIdx.x % NTD;
  const int jb = dtid / NIB, ib = dtid % NIB;
  bool first_tile = true;

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
    const int nsub = (nst + sub - 1) / sub;
    if (warp_active) {
      // the segment's checkpoint and controls
#pragma unroll
      for (int q = 0; q < SPW; ++q) {
        if (lane < 7) xs[q][lane] = act[q] ? __ldg(a.ckpt + ((size_t)kq[q] * n_ck + seg) * 7 + lane) : 0.0f;
        if (lane < nst) {
          const int t = t0 + lane;
          const float2 e = noise_at(p, (uint32_t)kq[q], (uint32_t)t);
          const float v0 = impq[q] ? __ldg(p.U + 2 * t) + e.x : e.x;
          const float v1 = impq[q] ? __ldg(p.U + 2 * t + 1) + e.y : e.y;
          *reinterpret_cast<float4 *>(vg[q] + 4 * lane) =
              make_float4(v0, v1, fminf(fmaxf(v0, p.umin0), p.umax0), fminf(fmaxf(v1, p.umin1), p.umax1));
        }
      }
      __syncwarp();
    }
    for (int b = nsub - 1; b >= 0; --b) {
      const int ib0 = b * sub, ie = min(ib0 + sub, nst);
      if (warp_active) {
        // (a) forward: the first pass runs the whole segment from the checkpoint (all states
        // kept); later passes re-run one sub-segment from its stored start state.  Rows of
        // h1 and h2 are kept for the sub-segment's steps only.
        const int i_start = b == nsub - 1 ? 0 : ib0;
        float x[SPW][7];
#pragma unroll
        for (int q = 0; q < SPW; ++q)
#pragma unroll
          for (int c = 0; c < 7; ++c) x[q][c] = xs[q][8 * i_start + c];
        for (int i = i_start; i < ie; ++i) {
          const int r = i >= ib0 ? i - ib0 : 0;  // row slot (rows before the sub-segment are scratch)
#pragma unroll
          for (int q = 0; q < SPW; ++q) {
            const float z[6] = {x[q][3], x[q][4], x[q][5], x[q][6], vg[q][4 * i + 2], vg[q][4 * i + 3]};
            float h1v[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
              float acc = b1_s[i1 + m];
#pragma unroll
              for (int c = 0; c < 6; ++c) acc = fmaf(W1r[m][c], z[c], acc);
              h1v[m] = activation<ACT>(acc);
            }
            if constexpr (M == 2) {
              *reinterpret_cast<float2 *>(hs1[q] + r * H + i1) = make_float2(h1v[0], h1v[1]);
            } else {
              hs1[q][r * H + i1] = h1v[0];
            }
          }
          __syncwarp();
          float pa[R][SPW];
#pragma unroll
          for (int rr = 0; rr < R; ++rr)
#pragma unroll
            for (int q = 0; q < SPW; ++q) pa[rr][q] = 0.0f;
#pragma unroll 4
          for (int ii = 0; ii < HH; ii += 4) {
            float4 hv[SPW];
#pragma unroll
            for (int q = 0; q < SPW; ++q) hv[q] = *reinterpret_cast<const float4 *>(hs1[q] + r * H + HH * ch + ii);
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
              const float4 w = *reinterpret_cast<const float4 *>(W2_s + (r4 + 16 * rr) * WS + HH * ch + ii);
#pragma unroll
              for (int q = 0; q < SPW; ++q) {
                pa[rr][q] = fmaf(w.x, hv[q].x, pa[rr][q]);
                pa[rr][q] = fmaf(w.y, hv[q].y, pa[rr][q]);
                pa[rr][q] = fmaf(w.z, hv[q].z, pa[rr][q]);
                pa[rr][q] = fmaf(w.w, hv[q].w, pa[rr][q]);
              }
            }
          }
          // rows r4 + 16 (ch + 2 m) = lane + 32 m stay; the partner's half arrives by shuffle
          float acc2[SPW][M];
#pragma unroll
          for (int m = 0; m < M; ++m)
#pragma unroll
            for (int q = 0; q < SPW; ++q) {
              const float mine = ch ? pa[2 * m + 1][q] : pa[2 * m][q];
              const float send = ch ? pa[2 * m][q] : pa[2 * m + 1][q];
              acc2[q][m] = b2_s[lane + 32 * m] + (mine + __shfl_xor_sync(FULL_MASK, send, 16));
            }
          __syncwarp();  // the row slot is rewritten by the next step when r is the scratch slot
#pragma unroll
          for (int q = 0; q < SPW; ++q) {
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int m = 0; m < M; ++m) {
              const float h2 = activation<ACT>(acc2[q][m]);
              hs2[q][r * H + lane + 32 * m] = h2;
              const float4 w3 = *reinterpret_cast<const float4 *>(W3_s + 4 * (lane + 32 * m));
              d[0] = fmaf(w3.x, h2, d[0]);
              d[1] = fmaf(w3.y, h2, d[1]);
              d[2] = fmaf(w3.z, h2, d[2]);
              d[3] = fmaf(w3.w, h2, d[3]);
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) d[o] = warp_sum(d[o]) + __ldg(net + net_off_b3(H) + o);
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
            float xl = x[q][0];
#pragma unroll
            for (int c = 1; c < 7; ++c) xl = lane == c ? x[q][c] : xl;
            if (lane < 7) xs[q][8 * (i + 1) + lane] = xl;
          }
        }
        __syncwarp();
        // (b) on the first pass: cost slopes at x_{t0+1 .. t0+nst}, one step per lane, and the
        // Sbar-weighted components
        if (b == nsub - 1) {
          float gcw[4] = {0.0f, 0.0f, 0.0f, 0.0f};
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
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const float c = warp_sum(gcw[o]);
            if (lane == 0) wsum_s[8 * warp + 4 + o] += c;
          }
        }
        __syncwarp();
        // (c) reverse the sub-segment's steps
        for (int i = ie - 1; i >= ib0; --i) {
          const int t = t0 + i;  // step t -> t + 1 used v_t
          const int r = i - ib0;
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
            for (int o = 0; o < 4; ++o) db[q][o] = dt * xb[q][3 + o];
#pragma unroll
            for (int m = 0; m < M; ++m) {
              const float h2 = hs2[q][r * H + lane + 32 * m];
              const float4 w3 = *reinterpret_cast<const float4 *>(W3_s + 4 * (lane + 32 * m));
              float hb = w3.x * db[q][0];
              hb = fmaf(w3.y, db[q][1], hb);
              hb = fmaf(w3.z, db[q][2], hb);
              hb = fmaf(w3.w, db[q][3], hb);
#pragma unroll
              for (int o = 0; o < 4; ++o) gW3[m][o] = fmaf(db[q][o], h2, gW3[m][o]);
              const float a2b = ACT == 1 ? hb : hb * (1.0f - h2 * h2);
              gb2[m] += a2b;
              hs2[q][r * H + lane + 32 * m] = a2b;
            }
          }
          if (lane == 0) {
#pragma unroll
            for (int o = 0; o < 4; ++o) wsum_s[8 * warp + o] += db[0][o] + db[1][o];
          }
          __syncwarp();
          float pb[CW][SPW];
#pragma unroll
          for (int cc = 0; cc < CW; ++cc)
#pragma unroll
            for (int q = 0; q < SPW; ++q) pb[cc][q] = 0.0f;
#pragma unroll 2
          for (int jj = 0; jj < HH; jj += 4) {
            float4 av[SPW];
#pragma unroll
            for (int q = 0; q < SPW; ++q) av[q] = *reinterpret_cast<const float4 *>(hs2[q] + r * H + HH * ch + jj);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const float *wrow = W2_s + (HH * ch + jj + kk) * WS + CW * r4;
              float wv[CW];
              if constexpr (CW == 4) {
                const float4 w = *reinterpret_cast<const float4 *>(wrow);
                wv[0] = w.x; wv[1] = w.y; wv[2] = w.z; wv[3] = w.w;
              } else {
                const float2 w = *reinterpret_cast<const float2 *>(wrow);
                wv[0] = w.x; wv[1] = w.y;
              }
#pragma unroll
              for (int q = 0; q < SPW; ++q) {
                const float a = kk == 0 ? av[q].x : kk == 1 ? av[q].y : kk == 2 ? av[q].z : av[q].w;
#pragma unroll
                for (int cc = 0; cc < CW; ++cc) pb[cc][q] = fmaf(wv[cc], a, pb[cc][q]);
              }
            }
          }
          // columns CW r4 + M ch + m stay; the partner's half arrives by shuffle
          float h1b[SPW][M];
#pragma unroll
          for (int m = 0; m < M; ++m)
#pragma unroll
            for (int q = 0; q < SPW; ++q) {
              const float mine = ch ? pb[M + m][q] : pb[m][q];
              const float send = ch ? pb[m][q] : pb[M + m][q];
              h1b[q][m] = mine + __shfl_xor_sync(FULL_MASK, send, 16);
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
              const float h1 = hs1[q][r * H + i1 + m];
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
            *reinterpret_cast<float2 *>(ub_w + 2 * t) = make_float2(ub[0], ub[1]);
          }
        }
      }
      __syncthreads();
      // (d) W2 gradient: sum over this CTA's active samples and the sub-segment's steps of
      // a2bar h1^T, added to the thread's tile of the record (first tile: stored)
      float gW2[TJ][TI];
#pragma unroll
      for (int rr = 0; rr < TJ; ++rr)
#pragma unroll
        for (int c = 0; c < TI; ++c) gW2[rr][c] = 0.0f;
      const int nrow = ie - ib0;
      const int s_lo = dhalf < 2 ? dhalf * NW : SC, s_hi = dhalf == 0 ? NW : SC;
      for (int sidx = s_lo; sidx < s_hi; ++sidx) {
        const int ks = blockIdx.x * SC + sidx;
        if (ks >= K || __ldg(a.w + ks) == 0.0f) continue;
        const float *h1w = sreg + sidx * sf + 8 * (every + 1) + 8 * every;
        const float *a2w = h1w + H * sub;
        for (int i = 0; i < nrow; ++i) {
          float ar[TJ];
          if constexpr (TJ == 4) {
            const float4 av = *reinterpret_cast<const float4 *>(a2w + i * H + TJ * jb);
            ar[0] = av.x; ar[1] = av.y; ar[2] = av.z; ar[3] = av.w;
          } else {
            const float2 av = *reinterpret_cast<const float2 *>(a2w + i * H + TJ * jb);
            ar[0] = av.x; ar[1] = av.y;
          }
          float hr[TI];
          if constexpr (TI == 2) {
            const float2 hv = *reinterpret_cast<const float2 *>(h1w + i * H + TI * ib);
            hr[0] = hv.x; hr[1] = hv.y;
          } else {
#pragma unroll
            for (int g = 0; g < TI / 4; ++g) {
              const float4 hv = *reinterpret_cast<const float4 *>(h1w + i * H + 4 * ib + 4 * NIB * g);
              hr[4 * g] = hv.x; hr[4 * g + 1] = hv.y; hr[4 * g + 2] = hv.z; hr[4 * g + 3] = hv.w;
            }
          }
#pragma unroll
          for (int rr = 0; rr < TJ; ++rr)
#pragma unroll
            for (int c = 0; c < TI; ++c) gW2[rr][c] = fmaf(ar[rr], hr[c], gW2[rr][c]);
        }
      }
      for (int turn = 0; turn < 2; ++turn) {
        if (turn == 1) __syncthreads();
        if (dhalf != turn) continue;
        const bool store = first_tile && turn == 0;
#pragma unroll
        for (int rr = 0; rr < TJ; ++rr) {
          float *dst = rec + net_off_W2(H) + (TJ * jb + rr) * H;
          if constexpr (TI == 2) {
            float2 *d2 = reinterpret_cast<float2 *>(dst + TI * ib);
            float2 v = make_float2(gW2[rr][0], gW2[rr][1]);
            if (!store) {
              const float2 o = *d2;
              v.x += o.x;
              v.y += o.y;
            }
            *d2 = v;
          } else {
#pragma unroll
            for (int g = 0; g < TI / 4; ++g) {
              float4 *d4 = reinterpret_cast<float4 *>(dst + 4 * ib + 4 * NIB * g);
              float4 v = make_float4(gW2[rr][4 * g], gW2[rr][4 * g + 1], gW2[rr][4 * g + 2], gW2[rr][4 * g + 3]);
              if (!store) {
                const float4 o = *d4;
                v.x += o.x;
                v.y += o.y;
                v.z += o.z;
                v.w += o.w;
              }
              *d4 = v;
            }
          }
        }
      }
      first_tile = false;
      __syncthreads();
    }
  }

  // ---- this CTA's record (the per-sample regions are free now): per-warp accumulators
  // summed in warp order; the W2 part is already in place ----
  float *rec_s = sreg;
  const int nf = net_floats(H);
  for (int e = threadIdx.x; e < nrec; e += NT) rec_s[e] = 0.0f;
  __syncthreads();
  for (int w = 0; w < NW; ++w) {
    if (warp == w) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j = lane + 32 * m;
#pragma unroll
        for (int c = 0; c < 6; ++c) rec_s[net_off_W1(H) + (i1 + m) * 6 + c] += gW1[m][c];
        rec_s[net_off_b1(H) + i1 + m] += gb1[m];
        rec_s[net_off_b2(H) + j] += gb2[m];
#pragma unroll
        for (int o = 0; o < 4; ++o) rec_s[net_off_W3(H) + o * H + j] += gW3[m][o];
      }
      // b3 and the cost multipliers (the Sbar-weighted components)
      if (lane < 4) {
        rec_s[net_off_b3(H) + lane] += wsum_s[8 * w + lane];
        rec_s[nf + lane] += wsum_s[8 * w + 4 + lane];
      }
    }
    __syncthreads();
  }
  // warps with an active sample wrote their dL/dU rows
  unsigned wmask = 0;
  for (int w = 0; w < NW; ++w)
#pragma unroll
    for (int q = 0; q < SPW; ++q) {
      const int k = blockIdx.x * SC + w * SPW + q;
      if (k < K && __ldg(a.w + k) != 0.0f) wmask |= 1u << w;
    }
  for (int e = threadIdx.x; e < 2 * T; e += NT) {
    float sum = 0.0f;
    for (int w = 0; w < NW; ++w)
      if (wmask >> w & 1u) sum += rec[nrec + (size_t)w * 2 * T + e];
    rec_s[nf + 4 + e] = sum;
  }
  __syncthreads();
  const int w2_lo = net_off_W2(H), w2_hi = w2_lo + H * H;
  for (int e = threadIdx.x; e < nrec; e += NT)
    if (e < w2_lo || e >= w2_hi) rec[e] = rec_s[e];
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
cudaError_t launch_bwd(const AdjParams &a, const AdjPlan &pl, cudaStream_t s) {
  auto kern = adj_backward_kernel<H, ACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  kern<<<pl.n_cta, pl.nw * 32, pl.smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

AdjPlan adj_plan(int K, int H, int every, int T, int n_sm, size_t smem_max) {
  AdjPlan pl;
  pl.nw = adj_warps(K, n_sm > 0 ? n_sm : 1);
  pl.n_cta = (K + kAdjSPW * pl.nw - 1) / (kAdjSPW * pl.nw);
  pl.sub = adj_sub_len(H, every, T, pl.nw, smem_max);
  pl.smem = sizeof(float) * adj_smem_floats(H, every, pl.sub, T, pl.nw);
  return pl;
}

// Any plan for K <= K_cap: at most ceil(K_cap / 16) CTAs (8 warps or more each), and
// n_cta * nw <= K_cap / 2 + 16 dL/dU rows.
size_t adj_part_floats(int K_cap, int H, int T_max) {
  const size_t n_cta = (K_cap + 2 * kAdjMinWarps - 1) / (2 * kAdjMinWarps);
  return n_cta * adj_rec_floats(H, T_max) + ((size_t)K_cap / 2 + kAdjMaxWarps) * 2 * T_max;
}

cudaError_t adj_launch_scalars(int K, int T, int n_imp, const float *w, const float *S, const float *Uo,
                               const float *gUo, const float *gJ, float *scal, float *J_out, cudaStream_t s) {
  adj_scalars_kernel<<<1, 1024, 0, s>>>(K, T, n_imp, w, S, Uo, gUo, gJ, scal, J_out);
  return cudaGetLastError();
}

cudaError_t adj_launch_backward(const AdjParams &a_in, const AdjPlan &pl, float *g_cost_w, float *g_U, float *g_net,
                                cudaStream_t s) {
  AdjParams a = a_in;
  const int H = a.p.H, T = a.p.T;
  a.sub = pl.sub;
  cudaError_t e;
  if (H == 32) e = a.p.activation == 1 ? launch_bwd<32, 1>(a, pl, s) : launch_bwd<32, 0>(a, pl, s);
  else if (H == 64) e = a.p.activation == 1 ? launch_bwd<64, 1>(a, pl, s) : launch_bwd<64, 0>(a, pl, s);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  const int nf = net_floats(H);
  const int n_out = nf + 4 + 2 * T;
  adj_reduce_kernel<<<(n_out + 31) / 32, 256, 0, s>>>(pl.n_cta, (int)adj_cta_floats(H, T, pl.nw), nf, T, a.part,
                                                      a.gUo, a.scal, g_net, g_cost_w, g_U);
  return cudaGetLastError();
}

}  // namespace itmpc
