// iterate_tps.cu -- thread-per-sample FP32 IT-MPC iterations for many samples:
// a single instance with large K, or many independent instances in one launch.
//
// One thread rolls out one sample (Alg. 1, inner loop) through the whole
// network of Sec. V-B: the weights live in the kernel parameter space, so
// every FMA reads its weight straight from the constant bank and nothing is
// broadcast through shared memory; each layer offers H independent FMA
// chains per thread.  The thread draws its own noise (Philox + Box-Muller),
// integrates the kinematics and adds the running cost of Sec. V-C after every
// step, so a step needs no communication at all.  This wins when there are
// enough samples to keep every SM busy; at a few thousand samples the
// warp-per-sample kernel of iterate_fp32.cu is faster.
//
// Kernel 1 (persistent): CTAs pull work units -- NT (64, 128 or 256, the
// autotuned tile) consecutive samples of one instance, longest horizon first -- from a global counter and
// write one partial record per unit (rho_c, eta_c, ..., E_c: Alg. 2 shifted by
// the unit's own minimum).  Kernel 2: one CTA per instance merges that
// instance's records into U', the weights and the diagnostics (log-sum-exp
// merge of itmpc_merge.cuh) and resets the unit counter for the next launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "itmpc_device.cuh"
#include "itmpc_merge.cuh"
#include "itmpc_sum.cuh"
#include "itmpc_units.cuh"

namespace itmpc {

namespace {

template <class DYN>
struct TpsParams {
  TpsShared sh;
  DYN dyn;
};

// Weight pair (w[i], w[i + 1]) from the parameter space; i even, the array 8-byte aligned.
__device__ __forceinline__ unsigned long long wpair(const float *w, int i) {
  return *reinterpret_cast<const unsigned long long *>(w + i);
}

// d = W3 tanh(W2 tanh(W1 z + b1) + b2) + b3 for one sample, z = (x_d, g(v)).
template <int H, int ACT>
__device__ __forceinline__ void tps_network(const TpsNet<H> &N, float x0, float x1, float x2, float x3, float g0,
                                            float g1, float &d0, float &d1, float &d2, float &d3) {
  const unsigned long long zero = f2pack(0.0f, 0.0f);
  const unsigned long long z01 = f2pack(x0, x1), z23 = f2pack(x2, x3), z45 = f2pack(g0, g1);
  unsigned long long h1[H / 2];
#pragma unroll
  for (int j = 0; j < H; j += 2) {
    float a[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      unsigned long long acc = ffma2(wpair(N.W1, (j + q) * 6), z01, zero);
      acc = ffma2(wpair(N.W1, (j + q) * 6 + 2), z23, acc);
      acc = ffma2(wpair(N.W1, (j + q) * 6 + 4), z45, acc);
      const float2 r = f2unpack(acc);
      a[q] = activation<ACT>((r.x + N.b1[j + q]) + r.y);
    }
    h1[j / 2] = f2pack(a[0], a[1]);
  }
  unsigned long long h2[H / 2];
#pragma unroll
  for (int j = 0; j < H; j += 2) {
    float a[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      unsigned long long acc = ffma2(wpair(N.W2, (j + q) * H), h1[0], zero);
#pragma unroll
      for (int i = 2; i < H; i += 2) acc = ffma2(wpair(N.W2, (j + q) * H + i), h1[i / 2], acc);
      const float2 r = f2unpack(acc);
      a[q] = activation<ACT>((r.x + N.b2[j + q]) + r.y);
    }
    h2[j / 2] = f2pack(a[0], a[1]);
  }
  float d[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    unsigned long long acc = ffma2(wpair(N.W3, o * H), h2[0], zero);
#pragma unroll
    for (int i = 2; i < H; i += 2) acc = ffma2(wpair(N.W3, o * H + i), h2[i / 2], acc);
    const float2 r = f2unpack(acc);
    d[o] = (r.x + N.b3[o]) + r.y;
  }
  d0 = d[0]; d1 = d[1]; d2 = d[2]; d3 = d[3];
}

// The network of Sec. V-B, its weights in the kernel parameter space.
template <int H, int ACT>
struct MlpDyn {
  TpsNet<H> net;
  __device__ __forceinline__ void eval(float x0, float x1, float x2, float x3, float g0, float g1, float &d0,
                                       float &d1, float &d2, float &d3) const {
    tps_network<H, ACT>(net, x0, x1, x2, x3, g0, g1, d0, d1, d2, d3);
  }
};

template <class DYN, int NT>
__global__ void __maxnreg__(96) tps_rollout_kernel(const __grid_constant__ TpsParams<DYN> P) {
  constexpr int NWARP = NT / 32;
  constexpr int G = NT / 32;  // 32-sample groups of a unit
  const TpsShared &sh = P.sh;
  const DYN &dyn = P.dyn;
  __shared__ float U_s[2 * ITMPC_MAX_T_DEV];
  __shared__ float e_s[NT];
  __shared__ float red[NWARP][8];
  __shared__ int unit_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    __syncthreads();  // the previous unit is done with the shared buffers
    if (tid == 0) unit_s = (int)atomicAdd(sh.unit_counter, 1u);
    __syncthreads();
    const int u = unit_s;
    if (u >= sh.n_units) return;
    const TpsUnit un = sh.units[u];
    const TpsInstance &I = sh.inst[un.inst];
    const int K = I.K, T = I.T;
    for (int i = tid; i < 2 * T; i += NT) U_s[i] = __ldg(I.U + i);
    __syncthreads();

    const int k = un.k0 + tid;
    const bool live = k < K;
    const bool imp = (long long)I.k_base + k < I.n_imp;  // global index (sharded iterations)
    const float *map = sh.maps + (size_t)I.map * (size_t)sh.map_stride;
    CSum Sc;  // S_k = sum_t c_t, compensated
    if (live) {
      float px = __ldg(I.x0 + 0), py = __ldg(I.x0 + 1), th = __ldg(I.x0 + 2);
      float xd0 = __ldg(I.x0 + 3), xd1 = __ldg(I.x0 + 4), xd2 = __ldg(I.x0 + 5), xd3 = __ldg(I.x0 + 6);
      // states of instance 0 (x_t at t = 0, every, 2 every, ...), when asked for
      const bool dbg = sh.states_out != nullptr && un.inst == 0 && k < sh.n_states;
      const int every = sh.states_every > 0 ? sh.states_every : 1;
      float *st_o = dbg ? sh.states_out + (size_t)k * (T / every + 1) * 7 : nullptr;
      if (dbg) {
        st_o[0] = px; st_o[1] = py; st_o[2] = th; st_o[3] = xd0; st_o[4] = xd1; st_o[5] = xd2; st_o[6] = xd3;
      }
      for (int t = 0; t < T; ++t) {
        const float2 e = tps_noise(sh, I.k_base + (uint32_t)k, (uint32_t)t, I.ctr2, I.ctr3);
        const float u0 = U_s[2 * t], u1 = U_s[2 * t + 1];
        const float v0 = imp ? u0 + e.x : e.x, v1 = imp ? u1 + e.y : e.y;
        const float g0 = fminf(fmaxf(v0, sh.umin0), sh.umax0), g1 = fminf(fmaxf(v1, sh.umin1), sh.umax1);
        // f(x_d, g(v)): 6 -> H -> H -> 4 with weights from the constant bank, two
        // products per instruction (packed FP32 pairs, even/odd partial sums)
        float d0, d1, d2, d3;
        dyn.eval(xd0, xd1, xd2, xd3, g0, g1, d0, d1, d2, d3);
        // explicit Euler from the old state (Sec. V-B)
        float sn, cs;
        sincosf(th, &sn, &cs);
        px = fmaf(cs * xd1 - sn * xd2, sh.dt, px);
        py = fmaf(sn * xd1 + cs * xd2, sh.dt, py);
        th = fmaf(xd3, sh.dt, th);
        xd0 = fmaf(d0, sh.dt, xd0);
        xd1 = fmaf(d1, sh.dt, xd1);
        xd2 = fmaf(d2, sh.dt, xd2);
        xd3 = fmaf(d3, sh.dt, xd3);
        if (dbg && (t + 1) % every == 0) {
          float *o = st_o + (size_t)((t + 1) / every) * 7;
          o[0] = px; o[1] = py; o[2] = th; o[3] = xd0; o[4] = xd1; o[5] = xd2; o[6] = xd3;
        }
        // running cost at x(t + 1) (Alg. 1) and the control-cost term (Sec. III-E)
        float c = tps_state_cost(sh, map, px, py, xd1, xd2, t + 1);
        if (sh.gamma != 0.0f) c += sh.gamma * (u0 * v0 * sh.inv_sig2_0 + u1 * v1 * sh.inv_sig2_1);
        Sc.add(c);
      }
      I.costs[k] = Sc.value();
    }
    const float S = Sc.value();

    // this unit's partial record (Alg. 2 shifted by the unit's own minimum)
    const bool fin = live && isfinite(S);
    float m = warp_min(fin ? S : INFINITY);
    if (lane == 0) red[warp][0] = m;
    __syncthreads();
    float rho = INFINITY;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) rho = fminf(rho, red[w][0]);
    const float e = (fin && isfinite(rho)) ? expf(-(S - rho) * sh.inv_lambda) : 0.0f;
    e_s[tid] = e;
    // compensated sums (itmpc_sum.cuh) over the warp, then over the warps
    CSum ce, ci, cq;
    ce.s = e;
    ci.s = imp && live ? e : 0.0f;
    cq.add_prod(e, e);
    ce = csum_warp(ce);
    ci = csum_warp(ci);
    cq = csum_warp(cq);
    const float nf = warp_sum(fin ? 1.0f : 0.0f);
    __syncthreads();  // every thread has read red[.][0]
    if (lane == 0) {
      red[warp][1] = ce.s; red[warp][2] = ce.c; red[warp][3] = ci.s; red[warp][4] = ci.c;
      red[warp][5] = cq.s; red[warp][6] = cq.c; red[warp][7] = nf;
    }
    __syncthreads();
    const int PL = partial_len(T);
    float *rec = sh.partials + I.rec_off + (size_t)un.idx * PL;
    if (tid == 0) {
      CSum a, b, c;
      float d = 0.f;
      for (int w = 0; w < NWARP; ++w) {
        a.add(CSum{red[w][1], red[w][2]});
        b.add(CSum{red[w][3], red[w][4]});
        c.add(CSum{red[w][5], red[w][6]});
        d += red[w][7];
      }
      rec[0] = rho; rec[1] = a.value(); rec[2] = b.value(); rec[3] = c.value(); rec[4] = d;
      rec[5] = 0.f; rec[6] = 0.f; rec[7] = 0.f;
    }
    // E_c[t] = sum_s e_s eps_s(t): item (t, group) sums 32 samples; the noise is
    // drawn again from its counter (samples with e = 0 are skipped); the G items
    // of one t sit on G consecutive lanes
    const int rounds = (G * T + NT - 1) / NT;
    for (int r = 0; r < rounds; ++r) {
      const int item = tid + r * NT;
      const bool valid = item < G * T;
      const int t = item / G, q = item % G;
      CSum a0, a1;
      if (valid) {
        for (int s2 = q * 32; s2 < q * 32 + 32; ++s2) {
          const float es = e_s[s2];
          if (es != 0.0f) {
            const float2 ep = tps_noise(sh, I.k_base + (uint32_t)(un.k0 + s2), (uint32_t)t, I.ctr2, I.ctr3);
            a0.add_prod(es, ep.x);
            a1.add_prod(es, ep.y);
          }
        }
      }
      a0 = csum_lanes(a0, G);
      a1 = csum_lanes(a1, G);
      if (valid && q == 0) {
        rec[8 + 2 * t] = a0.value();
        rec[8 + 2 * t + 1] = a1.value();
      }
    }
  }
}

constexpr int kMergeThreads = 256;

// CTA i < n_inst merges instance i.  With one instance and n_wcta > 0, CTAs n_inst ..
// n_inst + n_wcta - 1 write its K weights (each from the records' rho and eta) and CTA 0
// writes U', the stats and the status only.
__global__ void __launch_bounds__(kMergeThreads) tps_merge_kernel(const __grid_constant__ TpsShared sh,
                                                                  int stage_floats, int n_wcta) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  if (blockIdx.x == 0 && threadIdx.x == 0) *sh.unit_counter = 0u;  // the rollout kernel has finished
  const bool wcta = (int)blockIdx.x >= sh.n_inst;
  const TpsInstance &I = sh.inline_inst ? sh.inst0 : sh.inst[wcta ? 0 : blockIdx.x];
  IterParams q{};
  q.K = I.K;
  q.T = I.T;
  q.lambda = sh.lambda;
  q.inv_lambda = sh.inv_lambda;
  q.U = I.U;
  q.U_out = I.U_out;
  q.weights = I.weights;
  q.weights_inline = 1;
  q.costs = I.costs;
  q.stats = I.stats;
  q.status = sh.status;
  if (wcta) {
    merge_weights<kMergeThreads>(q, sh.partials + I.rec_off, I.n_units, (int)blockIdx.x - sh.n_inst, n_wcta);
    return;
  }
  if (n_wcta > 0) q.weights = nullptr;
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  __syncthreads();
  uint32_t phase = 0;
  merge_records<kMergeThreads>(q, sh.partials + I.rec_off, I.n_units, I.rec_out, reinterpret_cast<float *>(smem),
                               stage_floats, &mbar, phase);
}

template <class DYN, int NT>
cudaError_t tps_launch_d(const TpsParams<DYN> &P, int ctas_per_sm, cudaStream_t s) {
  const TpsShared &sh = P.sh;
  auto kern = tps_rollout_kernel<DYN, NT>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0)) != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
  const int grid = std::min(sh.n_units, per_sm * sms);
  kern<<<grid, NT, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace

__global__ void tps_advance_kernel(TpsInstance *inst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t it = (uint64_t)inst[i].ctr2 | ((uint64_t)(inst[i].ctr3 & 0xFFFFu) << 32);
  const uint64_t nx = (it + 1) & 0xFFFFFFFFFFFFull;
  inst[i].ctr2 = (uint32_t)nx;
  inst[i].ctr3 = (inst[i].ctr3 & 0xFFFF0000u) | (uint32_t)(nx >> 32);
}

cudaError_t tps_launch_advance(TpsInstance *inst, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  tps_advance_kernel<<<(n + 127) / 128, 128, 0, s>>>(inst, n);
  return cudaGetLastError();
}

size_t tps_merge_smem_bytes(int max_units_per_instance, int T_max) {
  const size_t n = (size_t)max_units_per_instance;
  return sizeof(float) * (((n + 3) & ~size_t(3)) + n * (size_t)partial_len(T_max) + 4);
}

cudaError_t tps_merge(const TpsShared &sh, cudaStream_t s) {
  // stage as many records as the device allows (the merge chunks the rest)
  int dev = 0, optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  size_t smem = 96 * 1024;
  if (smem > (size_t)optin) smem = (size_t)optin;
  static size_t configured[64] = {};
  if (dev >= 0 && dev < 64 && configured[dev] < smem) {
    if ((e = cudaFuncSetAttribute(tps_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    configured[dev] = smem;
  }
  // one instance: its weights are spread over CTAs of 2 x 256 samples each
  const int n_wcta = sh.n_inst == 1 && sh.single_K > 0 && sh.single_weights
                         ? std::min((sh.single_K + 2 * kMergeThreads - 1) / (2 * kMergeThreads), 148)
                         : 0;
  tps_merge_kernel<<<sh.n_inst + n_wcta, kMergeThreads, smem, s>>>(sh, (int)(smem / sizeof(float)), n_wcta);
  return cudaGetLastError();
}

template <class DYN>
cudaError_t tps_launch_nt(const TpsParams<DYN> &P, TpsTile tile, cudaStream_t s) {
  switch (tile.nt) {
    case 64: return tps_launch_d<DYN, 64>(P, tile.ctas_per_sm, s);
    case 128: return tps_launch_d<DYN, 128>(P, tile.ctas_per_sm, s);
    case 256: return tps_launch_d<DYN, 256>(P, tile.ctas_per_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int H, int ACT>
cudaError_t tps_launch_mlp(const TpsShared &sh, const float *net_host, TpsTile tile, cudaStream_t s) {
  TpsParams<MlpDyn<H, ACT>> P;
  P.sh = sh;
  // packed layout W1 [H][6], b1 [H], W2 [H][H], b2 [H], W3 [4][H], b3 [4] (== TpsNet field order)
  static_assert(sizeof(TpsNet<H>) == sizeof(float) * (size_t)net_floats(H), "network layout");
  memcpy(&P.dyn.net, net_host, sizeof(TpsNet<H>));
  return tps_launch_nt(P, tile, s);
}

cudaError_t tps_launch(const TpsShared &sh, const float *net_host, int H, int activation, TpsTile tile,
                       cudaStream_t s, const float *theta_host) {
  if (sh.n_units <= 0 || sh.n_inst <= 0) return cudaSuccess;
  cudaError_t e;
  if (theta_host) {
    TpsParams<BasisDyn> P;
    P.sh = sh;
    memcpy(P.dyn.theta, theta_host, sizeof(P.dyn.theta));
    e = tps_launch_nt(P, tile, s);
  } else {
    if (H != 32) return cudaErrorInvalidValue;  // the weights of wider networks do not fit the parameter space
    e = activation == 1 ? tps_launch_mlp<32, 1>(sh, net_host, tile, s) : tps_launch_mlp<32, 0>(sh, net_host, tile, s);
  }
  if (e != cudaSuccess) return e;
  return tps_merge(sh, s);
}

}  // namespace itmpc
