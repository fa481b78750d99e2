// iterate_wide.cu -- FP32 IT-MPC rollouts of the wide dynamics networks (6 -> H -> H -> 4,
// H = 64 or 128) for many samples: a single instance with large K, or a batch of instances.
//
// With H = 128 a sample-step of the network of Sec. V-B is 17.7 k multiply-adds, 93 % of
// them in the H x H hidden layer.  Spread over a tile of S samples that layer is a small
// GEMM per step, (S x H) x (H x H)^T, and this kernel computes it as one: a CTA owns S
// consecutive samples (one work unit) for the whole horizon, keeps W2 transposed in
// shared memory, and every thread accumulates a TS-sample x 4-neuron block of the
// product in registers, reading one float4 of activations and one float4 of weights per
// 4 TS FMAs.  A warp covers 8 neuron groups x 4 sample groups, so each of those loads is
// one shared-memory wavefront.  Per step (Alg. 1, inner loop):
//   warp 0, lane s   v = u + eps (noise drawn in blocks of kChunk steps into shared
//                    memory), g(v), the control-cost term, z = (x_d, g(v));
//   all threads      layer 1 (6-deep) and tanh  ->  h1^T [H][S];
//   all threads      layer 2 GEMM and tanh      ->  h2^T [H][S];
//   all threads      layer 3 partial sums (S samples x 4 outputs x P parts);
//   warp 0, lane s   x_d += dt f, Euler kinematics (Sec. V-B), and the running cost of
//                    Sec. V-C one step behind: the four texels of x_{t+1} are loaded
//                    now and used after the next step's GEMM, hiding their latency.
// The unit then writes the partial record of Alg. 2 (shifted by its own minimum) that
// tps_merge turns into U', the weights and the diagnostics -- the same records as the
// thread-per-sample and tensor-core kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "itmpc_device.cuh"
#include "itmpc_sum.cuh"
#include "itmpc_units.cuh"

namespace itmpc {

namespace {

template <int H>
struct WideShape;
template <>
struct WideShape<64> {
  static constexpr int S = 16, NT = 128, MIN_CTAS = 4;
};
template <>
struct WideShape<128> {
  static constexpr int S = 32, NT = 256, MIN_CTAS = 2;
};

constexpr int kChunk = 16;  // steps of noise drawn at a time

template <int H>
__host__ __device__ constexpr size_t wide_smem_floats(int T_max) {
  constexpr int S = WideShape<H>::S, NT = WideShape<H>::NT, P = NT / (4 * S);
  return (size_t)H * H + 6 * H + 2 * H + 4 * H + 4  // W2^T, W1^T, b1, b2, W3, b3 (padded)
         + 2 * (size_t)H * S                          // h1^T, h2^T
         + 8 * (size_t)S + (size_t)P * 4 * S           // z^T, layer-3 partials
         + 2 * (size_t)kChunk * S                       // noise block (float2)
         + (size_t)((2 * T_max + 3) & ~3) + (size_t)S;  // U, e
}

template <int H, int ACT>
__global__ void __launch_bounds__(WideShape<H>::NT, WideShape<H>::MIN_CTAS)
    wide_rollout_kernel(const __grid_constant__ TpsShared sh, const float *__restrict__ net) {
  constexpr int S = WideShape<H>::S, NT = WideShape<H>::NT;
  constexpr int NG = H / 4;               // groups of 4 neurons
  constexpr int TS = S * H / (NT * 4);    // samples per thread in the GEMM tile
  constexpr int SG = S / TS;              // groups of TS samples
  constexpr int NGW = 8, SGW = 4;         // one warp: 8 neuron groups x 4 sample groups
  constexpr int P = NT / (4 * S);         // layer-3 parts per (sample, output)
  static_assert(NG * SG == NT && NG % NGW == 0 && SG % SGW == 0, "tile");
  static_assert((NG / NGW) * (SG / SGW) == NT / 32 && P * 4 * S == NT && S <= 32, "shape");
  static_assert(TS == 2 || TS == 4, "vector width");

  extern __shared__ __align__(16) float sm[];
  float *W2T = sm;                 // [i][j] = W2[j][i]
  float *W1T = W2T + H * H;        // [m][j] = W1[j][m]
  float *b1s = W1T + 6 * H;
  float *b2s = b1s + H;
  float *W3s = b2s + H;            // [o][j]
  float *b3s = W3s + 4 * H;        // 4
  float *h1T = b3s + 4;            // [j][s]
  float *h2T = h1T + H * S;        // [j][s]
  float *zT = h2T + H * S;         // [m][s], m < 6 (8 rows)
  float *dp = zT + 8 * S;          // [part][o][s]
  float2 *eps_s = reinterpret_cast<float2 *>(dp + P * 4 * S);  // [chunk step][s]
  float *U_s = reinterpret_cast<float *>(eps_s + kChunk * S);
  float *e_s = U_s + ((2 * sh.T_max + 3) & ~3);
  __shared__ float red[5];
  __shared__ int unit_s;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < H * H; e += NT) {
    const int j = e / H, i = e % H;  // e = j H + i
    W2T[i * H + j] = __ldg(net + net_off_W2(H) + e);
  }
  for (int e = tid; e < 6 * H; e += NT) W1T[(e % 6) * H + e / 6] = __ldg(net + net_off_W1(H) + e);
  for (int e = tid; e < H; e += NT) {
    b1s[e] = __ldg(net + net_off_b1(H) + e);
    b2s[e] = __ldg(net + net_off_b2(H) + e);
  }
  for (int e = tid; e < 4 * H; e += NT) W3s[e] = __ldg(net + net_off_W3(H) + e);
  if (tid < 4) b3s[tid] = __ldg(net + net_off_b3(H) + tid);

  // this thread's GEMM tile: neurons 4 ng .. 4 ng + 3, samples TS sg .. TS sg + TS - 1
  const int ng = (warp % (NG / NGW)) * NGW + (lane % NGW);
  const int sg = (warp / (NG / NGW)) * SGW + (lane / NGW);
  // layer-3 role: sample s3, output o3, part p3
  const int s3 = tid % S, o3 = (tid / S) % 4, p3 = tid / (4 * S);
  const int every = sh.states_every > 0 ? sh.states_every : 1;

  for (;;) {
    __syncthreads();  // the previous unit is done with the shared buffers
    if (tid == 0) unit_s = (int)atomicAdd(sh.unit_counter, 1u);
    __syncthreads();
    const int u = unit_s;
    if (u >= sh.n_units) break;
    const TpsUnit un = sh.units[u];
    const TpsInstance &I = sh.inst[un.inst];
    const int K = I.K, T = I.T;
    for (int i = tid; i < 2 * T; i += NT) U_s[i] = __ldg(I.U + i);
    const float *map = sh.maps + (size_t)I.map * (size_t)sh.map_stride;

    // warp 0, lane s: the state of sample k = k0 + s
    const int k = un.k0 + lane;
    const bool owner = warp == 0 && lane < S;
    const bool live = owner && k < K;
    const bool imp = (long long)I.k_base + k < I.n_imp;  // global index (sharded iterations)
    const bool dbg = live && sh.states_out != nullptr && un.inst == 0 && k < sh.n_states;
    float px = 0.f, py = 0.f, th = 0.f, xd0 = 0.f, xd1 = 0.f, xd2 = 0.f, xd3 = 0.f;
    CSum Sacc;  // running cost over t, compensated
    // the pending running-cost lookup (texels of x_t loaded one step ahead)
    float pa = 0.f, pb = 0.f, m00 = 0.f, m01 = 0.f, m10 = 0.f, m11 = 0.f, pvx = 0.f, pvy = 0.f;
    if (owner) {
      px = __ldg(I.x0 + 0); py = __ldg(I.x0 + 1); th = __ldg(I.x0 + 2);
      xd0 = __ldg(I.x0 + 3); xd1 = __ldg(I.x0 + 4); xd2 = __ldg(I.x0 + 5); xd3 = __ldg(I.x0 + 6);
      if (dbg) {
        float *o = sh.states_out + (size_t)k * (T / every + 1) * 7;
        o[0] = px; o[1] = py; o[2] = th; o[3] = xd0; o[4] = xd1; o[5] = xd2; o[6] = xd3;
      }
    }

    for (int t = 0; t < T; ++t) {
      const int tc = t % kChunk;
      if (tc == 0) {
        __syncthreads();  // the previous block's noise has been used
        for (int item = tid; item < kChunk * S; item += NT) {
          const int s = item % S, tt = item / S;
          eps_s[item] = (t + tt < T) ? tps_noise(sh, I.k_base + (uint32_t)(un.k0 + s), (uint32_t)(t + tt), I.ctr2, I.ctr3)
                                     : make_float2(0.f, 0.f);
        }
        __syncthreads();
      }
      if (owner) {
        const float2 e = eps_s[tc * S + lane];
        const float u0 = U_s[2 * t], u1 = U_s[2 * t + 1];
        const float v0 = imp ? u0 + e.x : e.x, v1 = imp ? u1 + e.y : e.y;
        if (sh.gamma != 0.0f) Sacc.add(sh.gamma * (u0 * v0 * sh.inv_sig2_0 + u1 * v1 * sh.inv_sig2_1));
        zT[0 * S + lane] = xd0;
        zT[1 * S + lane] = xd1;
        zT[2 * S + lane] = xd2;
        zT[3 * S + lane] = xd3;
        zT[4 * S + lane] = fminf(fmaxf(v0, sh.umin0), sh.umax0);
        zT[5 * S + lane] = fminf(fmaxf(v1, sh.umin1), sh.umax1);
      }
      __syncthreads();

      // ---- layer 1: h1 = act(W1 z + b1) for this thread's tile ----
      {
        float zr[6][TS];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          if constexpr (TS == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(zT + m * S + 4 * sg);
            zr[m][0] = v.x; zr[m][1] = v.y; zr[m][2] = v.z; zr[m][3] = v.w;
          } else {
            const float2 v = *reinterpret_cast<const float2 *>(zT + m * S + 2 * sg);
            zr[m][0] = v.x; zr[m][1] = v.y;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * ng + q;
          float a[TS];
#pragma unroll
          for (int r = 0; r < TS; ++r) a[r] = b1s[j];
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const float w = W1T[m * H + j];
#pragma unroll
            for (int r = 0; r < TS; ++r) a[r] = fmaf(w, zr[m][r], a[r]);
          }
          if constexpr (TS == 4)
            *reinterpret_cast<float4 *>(h1T + j * S + 4 * sg) =
                make_float4(activation<ACT>(a[0]), activation<ACT>(a[1]), activation<ACT>(a[2]),
                            activation<ACT>(a[3]));
          else
            *reinterpret_cast<float2 *>(h1T + j * S + 2 * sg) =
                make_float2(activation<ACT>(a[0]), activation<ACT>(a[1]));
        }
      }
      __syncthreads();

      // ---- layer 2: (S x H) x (H x H)^T, one TS x 4 block per thread ----
      {
        float acc[TS][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float bq = b2s[4 * ng + q];
#pragma unroll
          for (int r = 0; r < TS; ++r) acc[r][q] = bq;
        }
#pragma unroll 8
        for (int i = 0; i < H; ++i) {
          const float4 w = *reinterpret_cast<const float4 *>(W2T + i * H + 4 * ng);
          float hv[TS];
          if constexpr (TS == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(h1T + i * S + 4 * sg);
            hv[0] = v.x; hv[1] = v.y; hv[2] = v.z; hv[3] = v.w;
          } else {
            const float2 v = *reinterpret_cast<const float2 *>(h1T + i * S + 2 * sg);
            hv[0] = v.x; hv[1] = v.y;
          }
#pragma unroll
          for (int r = 0; r < TS; ++r) {
            acc[r][0] = fmaf(hv[r], w.x, acc[r][0]);
            acc[r][1] = fmaf(hv[r], w.y, acc[r][1]);
            acc[r][2] = fmaf(hv[r], w.z, acc[r][2]);
            acc[r][3] = fmaf(hv[r], w.w, acc[r][3]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * ng + q;
          if constexpr (TS == 4)
            *reinterpret_cast<float4 *>(h2T + j * S + 4 * sg) =
                make_float4(activation<ACT>(acc[0][q]), activation<ACT>(acc[1][q]), activation<ACT>(acc[2][q]),
                            activation<ACT>(acc[3][q]));
          else
            *reinterpret_cast<float2 *>(h2T + j * S + 2 * sg) =
                make_float2(activation<ACT>(acc[0][q]), activation<ACT>(acc[1][q]));
        }
      }
      __syncthreads();

      // ---- layer 3 partial sums: d[s][o] over one part of the hidden units ----
      {
        constexpr int JP = H / P;
        float a0 = 0.f, a1 = 0.f;
        const float *w = W3s + o3 * H + p3 * JP;
        const float *h = h2T + (p3 * JP) * S + s3;
#pragma unroll 8
        for (int j = 0; j < JP; j += 2) {
          a0 = fmaf(w[j], h[j * S], a0);
          a1 = fmaf(w[j + 1], h[(j + 1) * S], a1);
        }
        dp[(p3 * 4 + o3) * S + s3] = a0 + a1;
      }
      __syncthreads();

      // ---- warp 0: Euler step (Sec. V-B), running cost one step behind (Sec. V-C) ----
      if (owner) {
        float d[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          float v = b3s[o];
#pragma unroll
          for (int p = 0; p < P; ++p) v += dp[(p * 4 + o) * S + lane];
          d[o] = v;
        }
        if (t > 0) {  // cost of x_t (loop index t) from the texels loaded last step
          float hh = (1.0f - pa) * (1.0f - pb) * m00 + pa * (1.0f - pb) * m01 + (1.0f - pa) * pb * m10 +
                     pa * pb * m11;
          Sacc.add(tps_cost_from_h(sh, hh, pvx, pvy, t));
        }
        float sn, cs;
        sincosf(th, &sn, &cs);
        px = fmaf(cs * xd1 - sn * xd2, sh.dt, px);
        py = fmaf(sn * xd1 + cs * xd2, sh.dt, py);
        th = fmaf(xd3, sh.dt, th);
        xd0 = fmaf(d[0], sh.dt, xd0);
        xd1 = fmaf(d[1], sh.dt, xd1);
        xd2 = fmaf(d[2], sh.dt, xd2);
        xd3 = fmaf(d[3], sh.dt, xd3);
        tps_costmap_fetch(sh, map, px, py, pa, pb, m00, m01, m10, m11);
        pvx = xd1;
        pvy = xd2;
        if (dbg && (t + 1) % every == 0) {
          float *o = sh.states_out + ((size_t)k * (T / every + 1) + (t + 1) / every) * 7;
          o[0] = px; o[1] = py; o[2] = th; o[3] = xd0; o[4] = xd1; o[5] = xd2; o[6] = xd3;
        }
      }
    }
    if (owner) {
      const float hh = (1.0f - pa) * (1.0f - pb) * m00 + pa * (1.0f - pb) * m01 + (1.0f - pa) * pb * m10 +
                       pa * pb * m11;
      Sacc.add(tps_cost_from_h(sh, hh, pvx, pvy, T));
      if (live) I.costs[k] = Sacc.value();
    }
    const float Sv = Sacc.value();

    // ---- this unit's partial record (Alg. 2 shifted by the unit's own minimum) ----
    if (warp == 0) {
      const bool fin = live && isfinite(Sv);
      const float rho = warp_min(fin ? Sv : INFINITY);
      const float e = (fin && isfinite(rho)) ? expf(-(Sv - rho) * sh.inv_lambda) : 0.0f;
      if (lane < S) e_s[lane] = e;
      CSum cq;
      cq.add_prod(e, e);
      const float eta = warp_csum(e), eta_imp = warp_csum(imp && live ? e : 0.0f);
      const float sq = csum_warp(cq).value(), nf = warp_sum(fin ? 1.0f : 0.0f);
      if (lane == 0) {
        red[0] = rho; red[1] = eta; red[2] = eta_imp; red[3] = sq; red[4] = nf;
      }
    }
    __syncthreads();
    const int PL = partial_len(T);
    float *rec = sh.partials + I.rec_off + (size_t)un.idx * PL;
    if (tid == 0) {
      rec[0] = red[0]; rec[1] = red[1]; rec[2] = red[2]; rec[3] = red[3]; rec[4] = red[4];
      rec[5] = 0.f; rec[6] = 0.f; rec[7] = 0.f;
    }
    // E_c[t] = sum_s e_s eps_s(t), the noise drawn again from its counter (e = 0 skipped)
    for (int t = tid; t < T; t += NT) {
      CSum a0, a1;
      for (int s = 0; s < S; ++s) {
        const float es = e_s[s];
        if (es != 0.0f) {
          const float2 ep = tps_noise(sh, I.k_base + (uint32_t)(un.k0 + s), (uint32_t)t, I.ctr2, I.ctr3);
          a0.add_prod(es, ep.x);
          a1.add_prod(es, ep.y);
        }
      }
      rec[8 + 2 * t] = a0.value();
      rec[8 + 2 * t + 1] = a1.value();
    }
  }
}

template <int H, int ACT>
cudaError_t wide_launch_h(const TpsShared &sh, const float *net, cudaStream_t s) {
  auto kern = wide_rollout_kernel<H, ACT>;
  const size_t smem = sizeof(float) * wide_smem_floats<H>(sh.T_max);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  // all of the unified L1 / shared array as shared memory, so that MIN_CTAS CTAs fit on an SM
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WideShape<H>::NT, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(sh.n_units, per_sm * sms);
  kern<<<grid, WideShape<H>::NT, smem, s>>>(sh, net);
  return cudaGetLastError();
}

}  // namespace

int wide_unit_samples(int H) { return H == 64 ? WideShape<64>::S : WideShape<128>::S; }

size_t wide_smem_bytes(int H, int T_max) {
  return sizeof(float) * (H == 64 ? wide_smem_floats<64>(T_max) : wide_smem_floats<128>(T_max));
}

cudaError_t wide_launch(const TpsShared &sh, const float *net, int H, int activation, cudaStream_t s) {
  if (sh.n_units <= 0 || sh.n_inst <= 0) return cudaSuccess;
  cudaError_t e;
  if (H == 64) e = activation == 1 ? wide_launch_h<64, 1>(sh, net, s) : wide_launch_h<64, 0>(sh, net, s);
  else if (H == 128) e = activation == 1 ? wide_launch_h<128, 1>(sh, net, s) : wide_launch_h<128, 0>(sh, net, s);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return tps_merge(sh, s);
}

}  // namespace itmpc
