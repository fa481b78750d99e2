// iterate_fp32.cu -- fused FP32 IT-MPC control iteration for sm_103a.
//
// One launch performs the whole iteration of Alg. 1 / Alg. 2:
//   phase 1  noise      eps for the CTA's samples x T steps, Philox + Box-Muller,
//                       kept in shared memory (never written to HBM);
//   phase 2  dynamics   the serial recurrence x_d(t+1) = x_d(t) + dt f(x_d(t), g(v_t))
//                       (Sec. V-B).  Only x_d feeds the network, so this is the
//                       only serial chain; a warp owns SPW samples, lane j owns
//                       hidden neuron j (+32, +64, ...), the hidden activations
//                       go through a per-warp shared buffer, W2 sits in registers
//                       when H = 32;
//   phase 3  kinematics the heading and position of Sec. V-B are prefix sums over t
//            and cost   of dt * theta_dot and dt * R(theta) v, evaluated with warp scans
//                       (lane = time step), followed by the state cost of Sec. V-C at
//                       every t = 1..T and the control-cost term of Sec. III-E;
//   phase 4  partials   per-CTA rho_c = min S, eta_c = sum e, E_c = sum e eps over the
//                       CTA's samples, with e = exp(-(S - rho_c)/lambda) (Alg. 2);
//   phase 5  combine    the last CTA to finish rescales every CTA's partials by
//                       exp(-(rho_c - rho)/lambda), forms U' (Sec. III-D), the
//                       weights, and diagnostics (log-sum-exp merge).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"

namespace itmpc {

namespace {

__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

struct SmemLayout {
  size_t U, eps, traj, W3, W2T, hbuf, S, e, total;
};

__host__ __device__ inline SmemLayout fp32_layout(int T, int H, int spw, int nwarps) {
  const int scta = spw * nwarps;
  SmemLayout L{};
  size_t off = 0;
  L.U = off;    off += align16(sizeof(float) * 2 * T);
  L.eps = off;  off += align16(sizeof(float2) * (size_t)scta * T);
  L.traj = off; off += align16(sizeof(float4) * (size_t)scta * (T + 1));
  L.W3 = off;   off += align16(sizeof(float) * (4 * (H + 4) + 4));
  L.W2T = off;  off += (H > 32) ? align16(sizeof(float) * (size_t)H * H) : 0;
  L.hbuf = off; off += align16(sizeof(float) * (size_t)nwarps * 2 * spw * H);
  L.S = off;    off += align16(sizeof(float) * scta);
  L.e = off;    off += align16(sizeof(float) * scta);
  L.total = off;
  return L;
}

template <int H, int SPW, int NWARPS>
__global__ void __launch_bounds__(NWARPS * 32) iterate_fp32_kernel(const __grid_constant__ IterParams p) {
  constexpr int NPL = H / 32;  // hidden neurons per lane
  constexpr int SCTA = SPW * NWARPS;
  constexpr bool W2_IN_REGS = (H == 32);
  constexpr int W3S = H + 4;  // padded row stride of W3 in shared memory

  extern __shared__ __align__(16) unsigned char smem[];
  const int T = p.T;
  const SmemLayout L = fp32_layout(T, H, SPW, NWARPS);
  float *U_s = reinterpret_cast<float *>(smem + L.U);
  float2 *eps_s = reinterpret_cast<float2 *>(smem + L.eps);
  float4 *traj_s = reinterpret_cast<float4 *>(smem + L.traj);
  float *W3_s = reinterpret_cast<float *>(smem + L.W3);
  float *W2T_s = reinterpret_cast<float *>(smem + L.W2T);
  float *hbuf = reinterpret_cast<float *>(smem + L.hbuf);
  float *S_s = reinterpret_cast<float *>(smem + L.S);
  float *e_s = reinterpret_cast<float *>(smem + L.e);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k0 = blockIdx.x * SCTA;
  const float *net = p.net;

  // ---- phase 0: nominal controls, output layer, (W2 transposed for H > 32) ----
  for (int i = tid; i < 2 * T; i += NWARPS * 32) U_s[i] = __ldg(p.U + i);
  for (int i = tid; i < 4 * H; i += NWARPS * 32) W3_s[(i / H) * W3S + (i % H)] = __ldg(net + net_off_W3(H) + i);
  if (tid < 4) W3_s[4 * W3S + tid] = __ldg(net + net_off_b3(H) + tid);
  if constexpr (!W2_IN_REGS) {
    for (int i = tid; i < H * H; i += NWARPS * 32) {
      const int j = i / H, k = i % H;  // W2[j][k] -> W2T[k][j]
      W2T_s[k * H + j] = __ldg(net + net_off_W2(H) + i);
    }
  }

  // ---- phase 1: noise for (s, t) of this CTA ----
  for (int i = tid; i < SCTA * T; i += NWARPS * 32) {
    const int s = i / T, t = i - s * T;
    const int k = k0 + s;
    float2 e = make_float2(0.0f, 0.0f);
    if (k < p.K) {
      e = noise_at(p, (uint32_t)k, (uint32_t)t);
      if (p.eps_out) reinterpret_cast<float2 *>(p.eps_out)[(size_t)k * T + t] = e;
    }
    eps_s[i] = e;
  }
  __syncthreads();

  // ---- phase 2: the serial network recurrence ----
  const int sw0 = warp * SPW;  // first sample of this warp within the CTA
  float xd[SPW][4];
  bool imp[SPW];
  const float x0r = __ldg(p.x0 + 3), x0vx = __ldg(p.x0 + 4), x0vy = __ldg(p.x0 + 5), x0w = __ldg(p.x0 + 6);
#pragma unroll
  for (int i = 0; i < SPW; ++i) {
    xd[i][0] = x0r; xd[i][1] = x0vx; xd[i][2] = x0vy; xd[i][3] = x0w;
    imp[i] = (k0 + sw0 + i) < p.n_imp;
  }
  if (lane < SPW) traj_s[(sw0 + lane) * (T + 1)] = make_float4(x0r, x0vx, x0vy, x0w);

  float w1[NPL][6], b1r[NPL], b2r[NPL];
  float w2[W2_IN_REGS ? NPL : 1][W2_IN_REGS ? H : 1];
#pragma unroll
  for (int n = 0; n < NPL; ++n) {
    const int j = lane + 32 * n;
#pragma unroll
    for (int q = 0; q < 6; ++q) w1[n][q] = __ldg(net + net_off_W1(H) + j * 6 + q);
    b1r[n] = __ldg(net + net_off_b1(H) + j);
    b2r[n] = __ldg(net + net_off_b2(H) + j);
    if constexpr (W2_IN_REGS) {
#pragma unroll
      for (int k = 0; k < H; ++k) w2[n][k] = __ldg(net + net_off_W2(H) + j * H + k);
    }
  }
  __syncthreads();  // W3_s, W2T_s ready

  float *h1buf = hbuf + warp * 2 * SPW * H;
  float *h2buf = h1buf + SPW * H;
  const int act = p.activation;
  const float dt = p.dt;

  for (int t = 0; t < T; ++t) {
    const float u0 = U_s[2 * t], u1 = U_s[2 * t + 1];
    float z[SPW][6];
#pragma unroll
    for (int i = 0; i < SPW; ++i) {
      const float2 e = eps_s[(sw0 + i) * T + t];
      const float v0 = imp[i] ? u0 + e.x : e.x;
      const float v1 = imp[i] ? u1 + e.y : e.y;
      z[i][0] = xd[i][0]; z[i][1] = xd[i][1]; z[i][2] = xd[i][2]; z[i][3] = xd[i][3];
      z[i][4] = fminf(fmaxf(v0, p.umin0), p.umax0);
      z[i][5] = fminf(fmaxf(v1, p.umin1), p.umax1);
    }
    // layer 1: 6 -> H
#pragma unroll
    for (int n = 0; n < NPL; ++n) {
#pragma unroll
      for (int i = 0; i < SPW; ++i) {
        float a = b1r[n];
#pragma unroll
        for (int q = 0; q < 6; ++q) a = fmaf(w1[n][q], z[i][q], a);
        h1buf[i * H + lane + 32 * n] = activation(a, act);
      }
    }
    __syncwarp();
    // layer 2: H -> H, h1 broadcast from shared memory
    float acc[NPL][SPW];
#pragma unroll
    for (int n = 0; n < NPL; ++n)
#pragma unroll
      for (int i = 0; i < SPW; ++i) acc[n][i] = b2r[n];
#pragma unroll
    for (int k = 0; k < H; k += 4) {
#pragma unroll
      for (int i = 0; i < SPW; ++i) {
        const float4 hv = *reinterpret_cast<const float4 *>(h1buf + i * H + k);
#pragma unroll
        for (int n = 0; n < NPL; ++n) {
          float wa, wb, wc, wd;
          if constexpr (W2_IN_REGS) {
            wa = w2[n][k]; wb = w2[n][k + 1]; wc = w2[n][k + 2]; wd = w2[n][k + 3];
          } else {
            const int j = lane + 32 * n;
            wa = W2T_s[k * H + j]; wb = W2T_s[(k + 1) * H + j];
            wc = W2T_s[(k + 2) * H + j]; wd = W2T_s[(k + 3) * H + j];
          }
          acc[n][i] = fmaf(wa, hv.x, acc[n][i]);
          acc[n][i] = fmaf(wb, hv.y, acc[n][i]);
          acc[n][i] = fmaf(wc, hv.z, acc[n][i]);
          acc[n][i] = fmaf(wd, hv.w, acc[n][i]);
        }
      }
    }
#pragma unroll
    for (int n = 0; n < NPL; ++n)
#pragma unroll
      for (int i = 0; i < SPW; ++i) h2buf[i * H + lane + 32 * n] = activation(acc[n][i], act);
    __syncwarp();
    // layer 3: H -> 4, lane 4i + o computes output o of sample i
    float d = 0.0f;
    if (lane < 4 * SPW) {
      const int i = lane >> 2, o = lane & 3;
      float a0 = W3_s[4 * W3S + o], a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
      for (int k = 0; k < H; k += 4) {
        const float4 hv = *reinterpret_cast<const float4 *>(h2buf + i * H + k);
        const float4 wv = *reinterpret_cast<const float4 *>(W3_s + o * W3S + k);
        a0 = fmaf(wv.x, hv.x, a0);
        a1 = fmaf(wv.y, hv.y, a1);
        a2 = fmaf(wv.z, hv.z, a2);
        a3 = fmaf(wv.w, hv.w, a3);
      }
      d = (a0 + a1) + (a2 + a3);
    }
#pragma unroll
    for (int i = 0; i < SPW; ++i) {
#pragma unroll
      for (int o = 0; o < 4; ++o) xd[i][o] = fmaf(__shfl_sync(FULL_MASK, d, 4 * i + o), dt, xd[i][o]);
      if (lane == i) traj_s[(sw0 + i) * (T + 1) + t + 1] = make_float4(xd[i][0], xd[i][1], xd[i][2], xd[i][3]);
    }
  }
  __syncwarp();

  // ---- phase 3: kinematics by prefix sums, then the running cost ----
  const float gamma = p.gamma;
  for (int i = 0; i < SPW; ++i) {
    const int s = sw0 + i;
    const int k = k0 + s;
    const bool is_imp = k < p.n_imp;
    float th_c = __ldg(p.x0 + 2), px_c = __ldg(p.x0 + 0), py_c = __ldg(p.x0 + 1);
    float Sacc = 0.0f;
    const bool dump = p.states_out != nullptr && k < p.n_states;
    if (dump && lane == 0) {
      float *o = p.states_out + (size_t)k * (T + 1) * 7;
      for (int q = 0; q < 7; ++q) o[q] = __ldg(p.x0 + q);
    }
    for (int base = 0; base < T; base += 32) {
      const int tau = base + lane;
      const bool valid = tau < T;
      const int tau_c = valid ? tau : T - 1;  // keep every shared-memory index in range
      float4 xo = traj_s[s * (T + 1) + tau_c];
      if (!valid) xo = make_float4(0.f, 0.f, 0.f, 0.f);
      const float dth = valid ? dt * xo.w : 0.0f;
      const float incl_th = warp_incl_scan(dth, lane);
      float excl_th = __shfl_up_sync(FULL_MASK, incl_th, 1);
      if (lane == 0) excl_th = 0.0f;
      const float th_old = th_c + excl_th;
      float sn, cs;
      sincosf(th_old, &sn, &cs);
      const float dpx = valid ? dt * (cs * xo.y - sn * xo.z) : 0.0f;
      const float dpy = valid ? dt * (sn * xo.y + cs * xo.z) : 0.0f;
      const float incl_px = warp_incl_scan(dpx, lane);
      const float incl_py = warp_incl_scan(dpy, lane);
      const float px = px_c + incl_px, py = py_c + incl_py, th = th_c + incl_th;
      if (valid) {
        const float4 xn = traj_s[s * (T + 1) + tau + 1];
        float c = state_cost(p, px, py, xn.y, xn.z, tau + 1);
        if (gamma != 0.0f) {
          const float2 e = eps_s[s * T + tau];
          const float u0 = U_s[2 * tau], u1 = U_s[2 * tau + 1];
          const float v0 = is_imp ? u0 + e.x : e.x, v1 = is_imp ? u1 + e.y : e.y;
          c += gamma * (u0 * v0 * p.inv_sig2_0 + u1 * v1 * p.inv_sig2_1);
        }
        Sacc += c;
        if (dump) {
          float *o = p.states_out + ((size_t)k * (T + 1) + tau + 1) * 7;
          o[0] = px; o[1] = py; o[2] = th; o[3] = xn.x; o[4] = xn.y; o[5] = xn.z; o[6] = xn.w;
        }
      }
      th_c += __shfl_sync(FULL_MASK, incl_th, 31);
      px_c += __shfl_sync(FULL_MASK, incl_px, 31);
      py_c += __shfl_sync(FULL_MASK, incl_py, 31);
    }
    const float S = warp_sum(Sacc);
    if (lane == 0) {
      S_s[s] = S;
      if (k < p.K) p.costs[k] = S;
    }
  }
  __syncthreads();

  // ---- phase 4: this CTA's partial sums ----
  float *rec = p.partials + (size_t)blockIdx.x * partial_len(T);
  if (warp == 0) {
    float m = INFINITY;
    for (int s = lane; s < SCTA; s += 32) {
      const float S = S_s[s];
      if (k0 + s < p.K && isfinite(S)) m = fminf(m, S);
    }
    m = warp_min(m);
    float eta = 0.f, eta_imp = 0.f, sq = 0.f, nf = 0.f;
    for (int s = lane; s < SCTA; s += 32) {
      const int k = k0 + s;
      const float S = S_s[s];
      const bool ok = k < p.K && isfinite(S) && isfinite(m);
      const float e = ok ? expf(-(S - m) * p.inv_lambda) : 0.0f;
      e_s[s] = e;
      eta += e;
      eta_imp += (k < p.n_imp) ? e : 0.0f;
      sq += e * e;
      nf += (k < p.K && isfinite(S)) ? 1.0f : 0.0f;
    }
    eta = warp_sum(eta); eta_imp = warp_sum(eta_imp); sq = warp_sum(sq); nf = warp_sum(nf);
    if (lane == 0) {
      rec[0] = m; rec[1] = eta; rec[2] = eta_imp; rec[3] = sq; rec[4] = nf;
      rec[5] = 0.f; rec[6] = 0.f; rec[7] = 0.f;
    }
  }
  __syncthreads();
  for (int o = tid; o < 2 * T; o += NWARPS * 32) {
    const float *ef = reinterpret_cast<const float *>(eps_s);
    float acc = 0.0f;
#pragma unroll 4
    for (int s = 0; s < SCTA; ++s) acc = fmaf(e_s[s], ef[(size_t)(s * T) * 2 + o], acc);
    rec[8 + o] = acc;
  }

  // ---- phase 5: the last CTA merges every CTA's partials ----
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) am_last = (atomicAdd(p.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();

  const int nC = gridDim.x;
  const int PL = partial_len(T);
  __shared__ float red[NWARPS][4];
  __shared__ float tot[4];
  float m = INFINITY;
  for (int c = tid; c < nC; c += NWARPS * 32) m = fminf(m, __ldcg(p.partials + (size_t)c * PL));
  m = warp_min(m);
  if (lane == 0) red[warp][0] = m;
  __syncthreads();
  if (tid == 0) {
    float r = INFINITY;
    for (int w = 0; w < NWARPS; ++w) r = fminf(r, red[w][0]);
    tot[0] = r;
  }
  __syncthreads();
  const float rho = tot[0];
  const bool ok = isfinite(rho);
  float eta = 0.f, eta_imp = 0.f, sq = 0.f, nf = 0.f;
  for (int c = tid; c < nC; c += NWARPS * 32) {
    const float *r = p.partials + (size_t)c * PL;
    const float rc = __ldcg(r);
    const float sc = (ok && isfinite(rc)) ? expf(-(rc - rho) * p.inv_lambda) : 0.0f;
    p.scale[c] = sc;
    eta += sc * __ldcg(r + 1);
    eta_imp += sc * __ldcg(r + 2);
    sq += sc * sc * __ldcg(r + 3);
    nf += __ldcg(r + 4);
  }
  eta = warp_sum(eta); eta_imp = warp_sum(eta_imp); sq = warp_sum(sq); nf = warp_sum(nf);
  __syncthreads();
  if (lane == 0) { red[warp][0] = eta; red[warp][1] = eta_imp; red[warp][2] = sq; red[warp][3] = nf; }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
    for (int w = 0; w < NWARPS; ++w) { a += red[w][0]; b += red[w][1]; c += red[w][2]; d += red[w][3]; }
    tot[0] = a; tot[1] = b; tot[2] = c; tot[3] = d;
  }
  __syncthreads();
  const float eta_t = tot[0], eta_imp_t = tot[1], sq_t = tot[2], nf_t = tot[3];
  const float inv_eta = ok ? 1.0f / eta_t : 0.0f;
  const float imp_frac = eta_imp_t * inv_eta;
  for (int o = tid; o < 2 * T; o += NWARPS * 32) {
    const float u = p.U[o];
    float out = u;
    if (ok) {
      // Neumaier-compensated sum over CTAs
      float sum = 0.0f, comp = 0.0f;
      for (int c = 0; c < nC; ++c) {
        const float term = __ldcg(p.scale + c) * __ldcg(p.partials + (size_t)c * PL + 8 + o);
        const float tsum = sum + term;
        comp += (fabsf(sum) >= fabsf(term)) ? (sum - tsum) + term : (term - tsum) + sum;
        sum = tsum;
      }
      out = u * imp_frac + (sum + comp) * inv_eta;
    }
    p.U_out[o] = out;
  }
  if (p.weights && p.weights_inline) {
    for (int k = tid; k < p.K; k += NWARPS * 32) {
      const float S = __ldcg(p.costs + k);
      p.weights[k] = (ok && isfinite(S)) ? expf(-(S - rho) * p.inv_lambda) * inv_eta : 0.0f;
    }
  }
  if (tid == 0) {
    p.stats[0] = rho;
    p.stats[1] = eta_t;
    p.stats[2] = ok ? eta_t * eta_t / sq_t : 0.0f;
    p.stats[3] = ok ? rho - p.lambda * logf(eta_t / (float)p.K) : INFINITY;
    p.stats[4] = nf_t;
    p.stats[5] = 0.f; p.stats[6] = 0.f; p.stats[7] = 0.f;
    if (!ok) *p.status = -3;  // ITMPC_ERR_NONFINITE
    *p.counter = 0u;          // ready for the next launch
  }
}

__global__ void finalize_weights_kernel(const __grid_constant__ IterParams p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.K) return;
  const float rho = p.stats[0], eta = p.stats[1];
  const float S = p.costs[k];
  p.weights[k] = (isfinite(rho) && isfinite(S)) ? expf(-(S - rho) * p.inv_lambda) / eta : 0.0f;
}

__global__ void noise_kernel(const __grid_constant__ IterParams p, float2 *eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)p.K * p.T) return;
  const int k = (int)(i / p.T), t = (int)(i - (int64_t)k * p.T);
  eps[i] = noise_at(p, (uint32_t)k, (uint32_t)t);
}

__global__ void philox_kernel(const uint4 *ctr, uint32_t k0, uint32_t k1, uint4 *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void tanh_kernel(const float *x, float *y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = tanh_f32(x[i]);
}

template <int H, int SPW, int NWARPS>
cudaError_t launch_tile(const IterParams &p, cudaStream_t s) {
  const SmemLayout L = fp32_layout(p.T, H, SPW, NWARPS);
  auto kern = iterate_fp32_kernel<H, SPW, NWARPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  const int nC = (p.K + SPW * NWARPS - 1) / (SPW * NWARPS);
  kern<<<nC, NWARPS * 32, L.total, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

Fp32Tile fp32_pick_tile(int K, int H) {
  (void)K;
  if (H == 128) return {2, 4};
  return {4, 4};
}

size_t fp32_smem_bytes(int T, int H, Fp32Tile t) { return fp32_layout(T, H, t.spw, t.nwarps).total; }

int fp32_num_ctas(int K, Fp32Tile t) { return (K + t.spw * t.nwarps - 1) / (t.spw * t.nwarps); }

cudaError_t fp32_launch_iterate(const IterParams &p, Fp32Tile tile, cudaStream_t s) {
#define ITMPC_TILE(HH, SS, WW) \
  if (p.H == HH && tile.spw == SS && tile.nwarps == WW) return launch_tile<HH, SS, WW>(p, s);
  ITMPC_TILE(32, 4, 4)
  ITMPC_TILE(64, 4, 4)
  ITMPC_TILE(128, 2, 4)
#undef ITMPC_TILE
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_finalize_weights(const IterParams &p, cudaStream_t s) {
  finalize_weights_kernel<<<(p.K + 255) / 256, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_noise(const IterParams &p, float *eps, cudaStream_t s) {
  const int64_t n = (int64_t)p.K * p.T;
  noise_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, reinterpret_cast<float2 *>(eps));
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4 *>(ctr), k0, k1,
                                                            reinterpret_cast<uint4 *>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_tanh(const float *x, float *y, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  tanh_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace itmpc
