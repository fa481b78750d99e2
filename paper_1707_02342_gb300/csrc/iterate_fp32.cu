// iterate_fp32.cu -- fused FP32 IT-MPC control iteration for sm_103a.
//
// One launch performs the whole iteration of Alg. 1 / Alg. 2.  A warp owns two
// samples (H = 32) or one (H = 64, 128); a CTA owns NW warps' consecutive samples.
//   phase 1  noise      eps and the clamped control g(v) for the CTA's samples x T
//                       steps (Philox-4x32-10 + Box-Muller), kept in shared memory;
//   phase 2  dynamics   the serial recurrence x_d(t+1) = x_d(t) + dt f(x_d(t), g(v_t))
//                       of Sec. V-B.  Only x_d feeds the network, so this is the one
//                       serial chain.  H = 32: a half-warp per sample, two neurons
//                       per lane, W2 rows in registers, the layer-1 pre-activation
//                       carried from step to step (recurrence_half32).  H = 64, 128:
//                       lane j owns neurons j, j + 32, ...; layer 1 in registers, h1
//                       broadcast through a per-warp shared row, W2 transposed in
//                       shared memory, the 4 outputs of layer 3 reduced across the
//                       warp with a register butterfly;
//   phase 3  kinematics heading and position are prefix sums over t of dt*theta_dot
//            and cost   and dt*R(theta)v (warp scans, lane = time step); then the state
//                       cost of Sec. V-C at t = 1..T plus the control-cost term of
//                       Sec. III-E, with every costmap load of a chunk in flight;
//   phase 4  partials   per-CTA rho_c = min S, eta_c = sum e, E_c = sum e eps with
//                       e = exp(-(S - rho_c)/lambda) (Alg. 2);
//   phase 5  combine    the last CTA of each group of CTAs merges the group's records
//                       (log-sum-exp rescaling by exp(-(rho_c - rho_g)/lambda)); the
//                       last group merger merges the group records into U' (Sec. III-D),
//                       the weights and the diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_merge.cuh"

namespace itmpc {

namespace {

__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

struct SmemLayout {
  size_t U, eps, gv, traj, pos, W2T, hbuf, W3b3, S, e, total;
};

__host__ __device__ inline SmemLayout fp32_layout(int T, int H, int nw, int spw) {
  const int scta = nw * spw;
  SmemLayout L{};
  size_t off = 0;
  L.U = off;    off += align16(sizeof(float) * 2 * T);
  L.eps = off;  off += align16(sizeof(float2) * (size_t)scta * T);
  L.gv = off;   off += align16(sizeof(float2) * (size_t)scta * T);
  L.traj = off; off += align16(sizeof(float4) * (size_t)scta * (T + 1));
  L.pos = off;  off += align16(sizeof(float4) * (size_t)scta * T);
  L.W2T = off;  off += (H > 32) ? align16(sizeof(float) * (size_t)H * H) : 0;
  L.hbuf = off; off += align16(sizeof(float) * (size_t)nw * (spw == 2 ? 2 * 32 * 36 + 16 + 80 : 2 * H));
  L.W3b3 = off; off += align16(sizeof(float) * (4 * H + 4));
  L.S = off;    off += align16(sizeof(float) * scta);
  L.e = off;    off += align16(sizeof(float) * scta);
  L.total = off;
  return L;
}

// ---- cooperative tail: a grid barrier, then every CTA merges a slice ----
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr uint32_t kBarrierPolls = 1u << 24;  // bounded wait: ~1 s of 64 ns sleeps

__device__ __forceinline__ unsigned atom_add_release_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid barrier for a cooperative launch (every CTA is resident).  Self-resetting:
// the last CTA to arrive zeroes the arrival count and bumps the generation the
// others poll.  `gen0` is the generation read by thread 0 any time before this
// CTA arrives.  The arrival is a release (orders the CTA's earlier global
// writes, made block-wide by the __syncthreads); the poll is an acquire.
// Returns false (and records ITMPC_ERR_TIMEOUT) if the wait ran out.
__device__ bool grid_barrier(const IterParams &p, unsigned gen0) {
  __shared__ int bar_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned *count = p.grid_bar, *gen = p.grid_bar + 1;
    int ok = 1;
    if (atom_add_release_u32(count, 1u) == gridDim.x - 1) {
      *count = 0u;  // read again only by the next launch, which starts after this one ends
      atom_add_release_u32(gen, 1u);
    } else {
      uint32_t i = 0;
      while (ld_acquire_u32(gen) == gen0) {
        if (++i > kBarrierPolls) {
          ok = 0;
          *p.status = kDevErrTimeout;
          break;
        }
        __nanosleep(32);
      }
    }
    bar_ok = ok;
  }
  __syncthreads();
  return bar_ok != 0;
}

// After the barrier: every CTA reads all record headers (rho_c, eta_c, ...),
// forms rho, eta and the per-record scales exactly as the tree merge does, writes
// the weights of its own samples and its slice of U'; CTA 0 writes the stats.
template <int NT, int SCTA>
__device__ void coop_tail(const IterParams &p, const float *S_s, int k0) {
  const int T = p.T, PL = partial_len(T), T2 = 2 * T, nC = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = NT / 32;
  constexpr int MAXS = 8;  // outputs per CTA slice at most
  __shared__ float red[NWARP][5 + MAXS];
  __shared__ float tot[5 + MAXS];
  const int per = (T2 + nC - 1) / nC;  // outputs per CTA (nC >= T2 / MAXS is checked on the host)
  const int o0 = blockIdx.x * per, on = max(0, min(per, T2 - o0));
  // every record this thread handles is read once (one round trip when nC <= NT)
  constexpr int MAXR = 2;  // records per thread kept in registers
  float4 hdr[MAXR];
  float nfr[MAXR], evr[MAXR][MAXS];
#pragma unroll
  for (int j = 0; j < MAXR; ++j) {
    const int c = tid + j * NT;
    hdr[j] = make_float4(INFINITY, 0.f, 0.f, 0.f);
    nfr[j] = 0.f;
#pragma unroll
    for (int q = 0; q < MAXS; ++q) evr[j][q] = 0.f;
    if (c < nC) {
      const float *r = p.partials + (size_t)c * PL;
      hdr[j] = __ldcg(reinterpret_cast<const float4 *>(r));
      nfr[j] = __ldcg(r + 4);
#pragma unroll
      for (int q = 0; q < MAXS; ++q)
        if (q < on) evr[j][q] = __ldcg(r + 8 + o0 + q);
    }
  }
  // pass 1: rho
  float m = INFINITY;
#pragma unroll
  for (int j = 0; j < MAXR; ++j) m = fminf(m, hdr[j].x);
  m = warp_min(m);
  if (lane == 0) red[warp][0] = m;
  __syncthreads();
  if (tid == 0) {
    float r = INFINITY;
    for (int w = 0; w < NWARP; ++w) r = fminf(r, red[w][0]);
    tot[0] = r;
  }
  __syncthreads();
  const float rho = tot[0];
  const bool ok = isfinite(rho);
  // pass 2: scalar sums and this CTA's E slice
  float acc[5 + MAXS];
#pragma unroll
  for (int q = 0; q < 5 + MAXS; ++q) acc[q] = 0.f;
#pragma unroll
  for (int j = 0; j < MAXR; ++j) {
    const float4 h = hdr[j];
    const float sc = (ok && isfinite(h.x)) ? expf(-(h.x - rho) * p.inv_lambda) : 0.0f;
    acc[0] += sc * h.y;
    acc[1] += sc * h.z;
    acc[2] += sc * sc * h.w;
    acc[3] += nfr[j];
#pragma unroll
    for (int q = 0; q < MAXS; ++q) acc[5 + q] = fmaf(sc, evr[j][q], acc[5 + q]);
  }
  __syncthreads();  // tot[0] consumed
#pragma unroll
  for (int q = 0; q < 5 + MAXS; ++q) {
    const float v = warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid < 5 + MAXS) {
    float a = 0.f;
    for (int w = 0; w < NWARP; ++w) a += red[w][tid];
    tot[tid] = a;
  }
  __syncthreads();
  const float eta = tot[0], eta_imp = tot[1], sq = tot[2], nf = tot[3];
  const float inv_eta = ok ? 1.0f / eta : 0.0f;
  if (tid < on) {
    const int o = o0 + tid;
    const float u = p.U[o];
    p.U_out[o] = ok ? u * (eta_imp * inv_eta) + tot[5 + tid] * inv_eta : u;
  }
  if (p.weights) {
    for (int q = tid; q < SCTA; q += NT) {
      const int k = k0 + q;
      if (k < p.K) {
        const float S = S_s[q];
        p.weights[k] = (ok && isfinite(S)) ? expf(-(S - rho) * p.inv_lambda) * inv_eta : 0.0f;
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    p.stats[0] = rho;
    p.stats[1] = eta;
    p.stats[2] = ok ? eta * eta / sq : 0.0f;
    p.stats[3] = ok ? rho - p.lambda * logf(eta / (float)p.K) : INFINITY;
    p.stats[4] = nf;
    p.stats[5] = 0.f; p.stats[6] = 0.f; p.stats[7] = 0.f;
    if (!ok) *p.status = kDevErrNonfinite;
  }
}

// Phase 2 for H = 32.  Layers 3 and 1 are affine, so with M = dt W1x W3
// (32 x 32), beta = dt W1x b3 and the Euler step x_d(t+1) = x_d(t) + dt d(t),
// d(t) = W3 h2(t) + b3, the input-layer pre-activation obeys
//   a1(t+1) = a1(t) + M h2(t) + beta + W1u (g(t+1) - g(t))
// (W1x, W1u: the state and control columns of W1; g the clamped control).
// The serial chain of a step is then two 32-term dot products with a tanh
// each, and x_d is not needed inside the loop: a1 is carried as a compensated
// (Kahan) sum, h2 rows go to a 32-step ring in shared memory (which is also the
// broadcast row of the M h2 product), and every 32 steps the output layer
// d = W3 h2 + b3 is applied to the whole block with lane = time step.  d(t) is
// left in traj[t + 1]; phase 3 turns it into x_d by prefix sums.
constexpr int kRingStride = 36;  // padded row: lanes reading rows t, t+1, .. hit distinct banks

// Two samples per warp: half-warp h = lane / 16 owns sample s_first + h and
// lane j = lane % 16 owns neurons j and j + 16 of it, so every activation
// broadcast feeds two FMAs per lane (half the shared-memory -> register traffic
// per sample-step of a one-neuron-per-lane layout).
// Per-warp buffer: ring 0 at 0, ring 1 at 32 rows + 16 floats (the other 16
// banks), then the two h1 rows at +0 and +48 floats: the halves' stores and
// loads never share a bank.
constexpr int kRing1 = 32 * kRingStride + 16;
constexpr int kHrows = kRing1 + 32 * kRingStride;
constexpr int kHalfWarpBuf = kHrows + 80;

template <int ACT>
__device__ __forceinline__ void recurrence_half32(const IterParams &p, const float *net, float *wbuf,
                                                  const float *W3b3_s, const float2 *gv_s, float4 *traj_s,
                                                  int s_first, int T, int lane) {
  constexpr int H = 32;
  const int h = lane >> 4, j = lane & 15;
  const int s = s_first + h;
  float *ring = wbuf + h * kRing1;
  float *hB = wbuf + kHrows + h * 48;
  const float4 *hB4 = reinterpret_cast<const float4 *>(hB);
  const float2 *gvr = gv_s + (size_t)s * T;
  float4 *traj = traj_s + (size_t)s * (T + 1);
  const float dt = p.dt;
  const int ja = j, jb = j + 16;
  float w1xa[4], w1xb[4], b3[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    w1xa[o] = __ldg(net + net_off_W1(H) + ja * 6 + o);
    w1xb[o] = __ldg(net + net_off_W1(H) + jb * 6 + o);
    b3[o] = W3b3_s[4 * H + o];
  }
  const float w1ua0 = __ldg(net + net_off_W1(H) + ja * 6 + 4), w1ua1 = __ldg(net + net_off_W1(H) + ja * 6 + 5);
  const float w1ub0 = __ldg(net + net_off_W1(H) + jb * 6 + 4), w1ub1 = __ldg(net + net_off_W1(H) + jb * 6 + 5);
  const float b2a = __ldg(net + net_off_b2(H) + ja), b2b = __ldg(net + net_off_b2(H) + jb);
  float beta_a = 0.f, beta_b = 0.f;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    beta_a = fmaf(dt * w1xa[o], b3[o], beta_a);
    beta_b = fmaf(dt * w1xb[o], b3[o], beta_b);
  }
  float ma[H], mb[H], w2a[H], w2b[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      a = fmaf(w1xa[o], W3b3_s[o * H + i], a);
      b = fmaf(w1xb[o], W3b3_s[o * H + i], b);
    }
    ma[i] = dt * a;
    mb[i] = dt * b;
    w2a[i] = __ldg(net + net_off_W2(H) + ja * H + i);
    w2b[i] = __ldg(net + net_off_W2(H) + jb * H + i);
  }
  // a1(0) = b1 + W1x x_d(0) + W1u g(0)
  float2 g = gvr[0];
  float a1a = __ldg(net + net_off_b1(H) + ja), a1b = __ldg(net + net_off_b1(H) + jb);
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float xo = __ldg(p.x0 + 3 + o);
    a1a = fmaf(w1xa[o], xo, a1a);
    a1b = fmaf(w1xb[o], xo, a1b);
  }
  a1a = fmaf(w1ua0, g.x, fmaf(w1ua1, g.y, a1a));
  a1b = fmaf(w1ub0, g.x, fmaf(w1ub1, g.y, a1b));
  float ca_c = 0.f, cb_c = 0.f;  // Kahan compensations
  for (int t = 0; t < T; ++t) {
    const float2 gn = gvr[t + 1 < T ? t + 1 : t];
    hB[ja] = activation<ACT>(a1a);
    hB[jb] = activation<ACT>(a1b);
    __syncwarp();
    float pa0 = b2a, pa1 = 0.f, pa2 = 0.f, pa3 = 0.f, pb0 = b2b, pb1 = 0.f, pb2 = 0.f, pb3 = 0.f;
#pragma unroll
    for (int kk = 0; kk < H; kk += 4) {
      const float4 hv = hB4[kk >> 2];
      pa0 = fmaf(w2a[kk], hv.x, pa0);
      pa1 = fmaf(w2a[kk + 1], hv.y, pa1);
      pa2 = fmaf(w2a[kk + 2], hv.z, pa2);
      pa3 = fmaf(w2a[kk + 3], hv.w, pa3);
      pb0 = fmaf(w2b[kk], hv.x, pb0);
      pb1 = fmaf(w2b[kk + 1], hv.y, pb1);
      pb2 = fmaf(w2b[kk + 2], hv.z, pb2);
      pb3 = fmaf(w2b[kk + 3], hv.w, pb3);
    }
    float *row = ring + (t & 31) * kRingStride;
    row[ja] = activation<ACT>((pa0 + pa1) + (pa2 + pa3));
    row[jb] = activation<ACT>((pb0 + pb1) + (pb2 + pb3));
    __syncwarp();
    if (t + 1 < T) {
      const float4 *row4 = reinterpret_cast<const float4 *>(row);
      const float dgx = gn.x - g.x, dgy = gn.y - g.y;
      float ea0 = fmaf(w1ua0, dgx, beta_a), ea1 = w1ua1 * dgy, ea2 = 0.f, ea3 = 0.f;
      float eb0 = fmaf(w1ub0, dgx, beta_b), eb1 = w1ub1 * dgy, eb2 = 0.f, eb3 = 0.f;
#pragma unroll
      for (int kk = 0; kk < H; kk += 4) {
        const float4 hv = row4[kk >> 2];
        ea0 = fmaf(ma[kk], hv.x, ea0);
        ea1 = fmaf(ma[kk + 1], hv.y, ea1);
        ea2 = fmaf(ma[kk + 2], hv.z, ea2);
        ea3 = fmaf(ma[kk + 3], hv.w, ea3);
        eb0 = fmaf(mb[kk], hv.x, eb0);
        eb1 = fmaf(mb[kk + 1], hv.y, eb1);
        eb2 = fmaf(mb[kk + 2], hv.z, eb2);
        eb3 = fmaf(mb[kk + 3], hv.w, eb3);
      }
      const float ya = ((ea0 + ea1) + (ea2 + ea3)) - ca_c;
      const float sa = a1a + ya;
      ca_c = (sa - a1a) - ya;
      a1a = sa;
      const float yb = ((eb0 + eb1) + (eb2 + eb3)) - cb_c;
      const float sb = a1b + yb;
      cb_c = (sb - a1b) - yb;
      a1b = sb;
      g = gn;
    }
    if ((t & 31) == 31 || t + 1 == T) {
      const int t0 = t & ~31;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int r = j + 16 * rr;
        if (t0 + r <= t) {
          const float4 *r4 = reinterpret_cast<const float4 *>(ring + r * kRingStride);
          float d0 = b3[0], d1 = b3[1], d2 = b3[2], d3 = b3[3];
#pragma unroll
          for (int kk = 0; kk < H; kk += 4) {
            const float4 hv = r4[kk >> 2];
            const float4 q0 = *reinterpret_cast<const float4 *>(W3b3_s + 0 * H + kk);
            const float4 q1 = *reinterpret_cast<const float4 *>(W3b3_s + 1 * H + kk);
            const float4 q2 = *reinterpret_cast<const float4 *>(W3b3_s + 2 * H + kk);
            const float4 q3 = *reinterpret_cast<const float4 *>(W3b3_s + 3 * H + kk);
            d0 = fmaf(q0.x, hv.x, fmaf(q0.y, hv.y, fmaf(q0.z, hv.z, fmaf(q0.w, hv.w, d0))));
            d1 = fmaf(q1.x, hv.x, fmaf(q1.y, hv.y, fmaf(q1.z, hv.z, fmaf(q1.w, hv.w, d1))));
            d2 = fmaf(q2.x, hv.x, fmaf(q2.y, hv.y, fmaf(q2.z, hv.z, fmaf(q2.w, hv.w, d2))));
            d3 = fmaf(q3.x, hv.x, fmaf(q3.y, hv.y, fmaf(q3.z, hv.z, fmaf(q3.w, hv.w, d3))));
          }
          traj[t0 + r + 1] = make_float4(d0, d1, d2, d3);
        }
      }
      __syncwarp();  // the ring is reused by the next block
    }
  }
}

template <int H, int NW, int SPW, int ACT>
__global__ void __launch_bounds__(NW * 32, 1) iterate_fp32_kernel(const __grid_constant__ IterParams p) {
  static_assert((SPW == 2) == (H == 32), "H = 32 runs two samples per warp, H = 64 / 128 one");
  constexpr int NT = NW * 32;
  constexpr int SCTA = NW * SPW;  // samples per CTA
  constexpr int NPL = H / 32;  // hidden neurons per lane

  extern __shared__ __align__(16) unsigned char smem[];
  const int T = p.T;
  const SmemLayout L = fp32_layout(T, H, NW, SPW);
  float *U_s = reinterpret_cast<float *>(smem + L.U);
  float2 *eps_s = reinterpret_cast<float2 *>(smem + L.eps);
  float2 *gv_s = reinterpret_cast<float2 *>(smem + L.gv);
  float4 *traj_s = reinterpret_cast<float4 *>(smem + L.traj);
  float4 *pos_s = reinterpret_cast<float4 *>(smem + L.pos);
  float *W2T_s = reinterpret_cast<float *>(smem + L.W2T);
  float *S_s = reinterpret_cast<float *>(smem + L.S);
  float *e_s = reinterpret_cast<float *>(smem + L.e);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k0 = blockIdx.x * SCTA;
  const float *net = p.net;

  // ---- phase 0/1: nominal controls, W3|b3, W2 transposed (H > 32), noise and g(v) ----
  float *W3b3_s = reinterpret_cast<float *>(smem + L.W3b3);
  unsigned gen0 = 0;
  if (p.coop && tid == 0) gen0 = ld_acquire_u32(p.grid_bar + 1);  // generation before this launch's barrier
  if (tid == 0 && (reinterpret_cast<uintptr_t>(p.map) & 15) == 0) {
    // bring this CTA's slice of the costmap into L2 while the rollouts run (phase 3 reads it)
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
  for (int i = tid; i < 4 * H + 4; i += NT) W3b3_s[i] = __ldg(net + net_off_W3(H) + i);  // W3 then b3
  if constexpr (H > 32) {
    for (int i = tid; i < H * H; i += NT) {
      const int j = i / H, kk = i - j * H;  // W2[j][kk] -> W2T[kk][j]
      W2T_s[kk * H + j] = __ldg(net + net_off_W2(H) + i);
    }
  }
  // counter words 2-3 of this iteration (plus the device-side offset of a replayed graph)
  uint32_t c2 = p.ctr2, c3 = p.ctr3;
  if (p.iter_add != nullptr) {
    const unsigned long long it =
        (((unsigned long long)(c3 & 0xFFFFu) << 32) | c2) + *p.iter_add;
    c2 = (uint32_t)it;
    c3 = (c3 & 0xFFFF0000u) | (uint32_t)((it >> 32) & 0xFFFFu);
  }
  for (int i = tid; i < SCTA * T; i += NT) {
    const int s = i / T, t = i - s * T;
    const int k = k0 + s;
    float2 e = make_float2(0.0f, 0.0f);
    if (k < p.K) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)t, c2, c3), p.key0, p.key1);
      const float2 z = box_muller(w.x, w.y);
      e = make_float2(p.sigma0 * z.x, p.sigma1 * z.y);
      if (p.eps_out) reinterpret_cast<float2 *>(p.eps_out)[(size_t)k * T + t] = e;
    }
    const bool imp = k < p.n_imp;
    const float v0 = imp ? __ldg(p.U + 2 * t) + e.x : e.x;
    const float v1 = imp ? __ldg(p.U + 2 * t + 1) + e.y : e.y;
    eps_s[i] = e;
    gv_s[i] = make_float2(fminf(fmaxf(v0, p.umin0), p.umax0), fminf(fmaxf(v1, p.umin1), p.umax1));
  }

  // per-lane network slices
  float w1[NPL][6], b1r[NPL], b2r[NPL], w3[NPL][4];
#pragma unroll
  for (int n = 0; n < NPL; ++n) {
    const int j = lane + 32 * n;
#pragma unroll
    for (int q = 0; q < 6; ++q) w1[n][q] = __ldg(net + net_off_W1(H) + j * 6 + q);
    b1r[n] = __ldg(net + net_off_b1(H) + j);
    b2r[n] = __ldg(net + net_off_b2(H) + j);
#pragma unroll
    for (int o = 0; o < 4; ++o) w3[n][o] = __ldg(net + net_off_W3(H) + o * H + j);
  }
  float b3r[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) b3r[o] = __ldg(net + net_off_b3(H) + o);
  __syncthreads();

  const float dt = p.dt;
  const float x0px = __ldg(p.x0 + 0), x0py = __ldg(p.x0 + 1), x0th = __ldg(p.x0 + 2);

  // ---- phase 2: the serial network recurrence ----
  if constexpr (SPW == 2) {
    float *wbuf = reinterpret_cast<float *>(smem + L.hbuf) + warp * kHalfWarpBuf;
    if ((lane & 15) == 0)
      traj_s[(warp * 2 + (lane >> 4)) * (T + 1)] =
          make_float4(__ldg(p.x0 + 3), __ldg(p.x0 + 4), __ldg(p.x0 + 5), __ldg(p.x0 + 6));
    recurrence_half32<ACT>(p, net, wbuf, W3b3_s, gv_s, traj_s, warp * 2, T, lane);
    __syncwarp();
  } else if (k0 + warp < p.K) {
    // H = 64 / 128: one warp per sample
    const int s = warp;
    float xd0 = __ldg(p.x0 + 3), xd1 = __ldg(p.x0 + 4), xd2 = __ldg(p.x0 + 5), xd3 = __ldg(p.x0 + 6);
    float *hrow = reinterpret_cast<float *>(smem + L.hbuf) + s * 2 * H;
    const float4 *hrow4 = reinterpret_cast<const float4 *>(hrow);
    float4 *traj = traj_s + s * (T + 1);
    const float2 *gvr = gv_s + s * T;
    if (lane == 0) traj[0] = make_float4(xd0, xd1, xd2, xd3);
    const int hi16 = (lane >> 4) & 1, hi8 = (lane >> 3) & 1;
    float2 g_next = gvr[0];
    for (int t = 0; t < T; ++t) {
      const float2 g = g_next;
      g_next = gvr[t + 1 < T ? t + 1 : t];  // next step's control, off the critical path
      // layer 1: 6 -> H
      __syncwarp();  // every lane has finished reading the previous h1 row
#pragma unroll
      for (int n = 0; n < NPL; ++n) {
        float a = b1r[n];
        a = fmaf(w1[n][0], xd0, a);
        a = fmaf(w1[n][1], xd1, a);
        a = fmaf(w1[n][2], xd2, a);
        a = fmaf(w1[n][3], xd3, a);
        a = fmaf(w1[n][4], g.x, a);
        a = fmaf(w1[n][5], g.y, a);
        hrow[lane + 32 * n] = activation<ACT>(a);
      }
      __syncwarp();
      // layer 2: H -> H, four independent chains per neuron
      float acc[NPL][4];
#pragma unroll
      for (int n = 0; n < NPL; ++n) {
        acc[n][0] = b2r[n]; acc[n][1] = 0.f; acc[n][2] = 0.f; acc[n][3] = 0.f;
      }
#pragma unroll
      for (int kk = 0; kk < H; kk += 4) {
        const float4 hv = hrow4[kk >> 2];
#pragma unroll
        for (int n = 0; n < NPL; ++n) {
          const int j = lane + 32 * n;
          const float wa = W2T_s[kk * H + j], wb = W2T_s[(kk + 1) * H + j];
          const float wc = W2T_s[(kk + 2) * H + j], wd = W2T_s[(kk + 3) * H + j];
          acc[n][0] = fmaf(wa, hv.x, acc[n][0]);
          acc[n][1] = fmaf(wb, hv.y, acc[n][1]);
          acc[n][2] = fmaf(wc, hv.z, acc[n][2]);
          acc[n][3] = fmaf(wd, hv.w, acc[n][3]);
        }
      }
      // layer 3 partial products of this lane's neurons
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
      for (int n = 0; n < NPL; ++n) {
        const float h2 = activation<ACT>((acc[n][0] + acc[n][1]) + (acc[n][2] + acc[n][3]));
        p0 = fmaf(w3[n][0], h2, p0);
        p1 = fmaf(w3[n][1], h2, p1);
        p2 = fmaf(w3[n][2], h2, p2);
        p3 = fmaf(w3[n][3], h2, p3);
      }
      // butterfly reduce-scatter of (p0..p3) over the warp: lane ends with output (lane >> 3) & 3
      const float s0 = hi16 ? p0 : p2, s1 = hi16 ? p1 : p3;
      const float q0 = (hi16 ? p2 : p0) + __shfl_xor_sync(FULL_MASK, s0, 16);
      const float q1 = (hi16 ? p3 : p1) + __shfl_xor_sync(FULL_MASK, s1, 16);
      float v = (hi8 ? q1 : q0) + __shfl_xor_sync(FULL_MASK, hi8 ? q0 : q1, 8);
      v += __shfl_xor_sync(FULL_MASK, v, 4);
      v += __shfl_xor_sync(FULL_MASK, v, 2);
      v += __shfl_xor_sync(FULL_MASK, v, 1);
      const float d0 = __shfl_sync(FULL_MASK, v, 0) + b3r[0];
      const float d1 = __shfl_sync(FULL_MASK, v, 8) + b3r[1];
      const float d2 = __shfl_sync(FULL_MASK, v, 16) + b3r[2];
      const float d3 = __shfl_sync(FULL_MASK, v, 24) + b3r[3];
      xd0 = fmaf(d0, dt, xd0);
      xd1 = fmaf(d1, dt, xd1);
      xd2 = fmaf(d2, dt, xd2);
      xd3 = fmaf(d3, dt, xd3);
      if (lane == 0) traj[t + 1] = make_float4(xd0, xd1, xd2, xd3);
    }
    __syncwarp();
  }

  // ---- phase 3: kinematics and running costs, this warp's samples side by side ----
  {
    float th_c[SPW], px_c[SPW], py_c[SPW];
    float4 xd_c[SPW];
#pragma unroll
    for (int q = 0; q < SPW; ++q) {
      th_c[q] = x0th;
      px_c[q] = x0px;
      py_c[q] = x0py;
      xd_c[q] = traj_s[(warp * SPW + q) * (T + 1)];
    }
    // 3a: x_d (H = 32: from the stored d), heading and position by prefix sums over t
    for (int base = 0; base < T; base += 32) {
      const int tau = base + lane;
      const bool valid = tau < T;
#pragma unroll
      for (int q = 0; q < SPW; ++q) {
        const int s = warp * SPW + q;
        float4 *traj = traj_s + s * (T + 1);
        float4 xo;
        if constexpr (H == 32) {
          // traj[tau + 1] holds d(tau): x_d(tau + 1) = x_d(0) + dt sum_{s <= tau} d(s)
          float4 dd = traj[valid ? tau + 1 : T];
          if (!valid) dd = make_float4(0.f, 0.f, 0.f, 0.f);
          const float i0 = warp_incl_scan(dt * dd.x, lane), i1 = warp_incl_scan(dt * dd.y, lane);
          const float i2 = warp_incl_scan(dt * dd.z, lane), i3 = warp_incl_scan(dt * dd.w, lane);
          // every lane takes part in each shuffle; lane 0 then drops the value
          float e0 = __shfl_up_sync(FULL_MASK, i0, 1), e1 = __shfl_up_sync(FULL_MASK, i1, 1);
          float e2 = __shfl_up_sync(FULL_MASK, i2, 1), e3 = __shfl_up_sync(FULL_MASK, i3, 1);
          if (lane == 0) e0 = e1 = e2 = e3 = 0.f;
          xo = make_float4(xd_c[q].x + e0, xd_c[q].y + e1, xd_c[q].z + e2, xd_c[q].w + e3);
          __syncwarp();  // every lane has read its d before any x_d overwrites it
          if (valid) traj[tau + 1] = make_float4(xd_c[q].x + i0, xd_c[q].y + i1, xd_c[q].z + i2, xd_c[q].w + i3);
          xd_c[q].x += __shfl_sync(FULL_MASK, i0, 31);
          xd_c[q].y += __shfl_sync(FULL_MASK, i1, 31);
          xd_c[q].z += __shfl_sync(FULL_MASK, i2, 31);
          xd_c[q].w += __shfl_sync(FULL_MASK, i3, 31);
        } else {
          xo = traj[valid ? tau : T - 1];
        }
        if (!valid) xo = make_float4(0.f, 0.f, 0.f, 0.f);
        const float dth = dt * xo.w;
        const float incl_th = warp_incl_scan(dth, lane);
        float excl_th = __shfl_up_sync(FULL_MASK, incl_th, 1);
        if (lane == 0) excl_th = 0.0f;
        float sn, cs;
        sincosf(th_c[q] + excl_th, &sn, &cs);
        const float dpx = dt * (cs * xo.y - sn * xo.z);
        const float dpy = dt * (sn * xo.y + cs * xo.z);
        const float incl_px = warp_incl_scan(dpx, lane);
        const float incl_py = warp_incl_scan(dpy, lane);
        if (valid) pos_s[s * T + tau] = make_float4(px_c[q] + incl_px, py_c[q] + incl_py, th_c[q] + incl_th, 0.f);
        th_c[q] += __shfl_sync(FULL_MASK, incl_th, 31);
        px_c[q] += __shfl_sync(FULL_MASK, incl_px, 31);
        py_c[q] += __shfl_sync(FULL_MASK, incl_py, 31);
      }
    }
    __syncwarp();

    // 3b: running cost at x(t), t = 1..T, plus the control-cost term
    const float gamma = p.gamma;
    float Sacc[SPW];
#pragma unroll
    for (int q = 0; q < SPW; ++q) Sacc[q] = 0.0f;
    for (int base = 0; base < T; base += 32) {
      const int tau = base + lane;
      if (tau < T) {
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
          const int s = warp * SPW + q;
          const int k = k0 + s;
          const float4 ps = pos_s[s * T + tau];
          const float4 xn = traj_s[s * (T + 1) + tau + 1];
          float c = state_cost(p, ps.x, ps.y, xn.y, xn.z, tau + 1);
          if (gamma != 0.0f) {
            const bool is_imp = k < p.n_imp;
            const float2 e = eps_s[s * T + tau];
            const float u0 = U_s[2 * tau], u1 = U_s[2 * tau + 1];
            const float v0 = is_imp ? u0 + e.x : e.x, v1 = is_imp ? u1 + e.y : e.y;
            c += gamma * (u0 * v0 * p.inv_sig2_0 + u1 * v1 * p.inv_sig2_1);
          }
          Sacc[q] += c;
          if (p.states_out != nullptr && k < p.n_states && (tau + 1) % p.states_every == 0) {
            float *o = p.states_out + ((size_t)k * (T / p.states_every + 1) + (tau + 1) / p.states_every) * 7;
            o[0] = ps.x; o[1] = ps.y; o[2] = ps.z; o[3] = xn.x; o[4] = xn.y; o[5] = xn.z; o[6] = xn.w;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < SPW; ++q) {
      const int s = warp * SPW + q;
      const int k = k0 + s;
      const float S = warp_sum(Sacc[q]);
      if (k < p.K) {
        if (p.states_out != nullptr && k < p.n_states && lane < 7)
          p.states_out[(size_t)k * (T / p.states_every + 1) * 7 + lane] = __ldg(p.x0 + lane);
        if (lane == 0) {
          S_s[s] = S;
          p.costs[k] = S;
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 4: this CTA's partial record ----
  float *rec = p.partials + (size_t)blockIdx.x * partial_len(T);
  if (warp == 0) {
    float m = INFINITY;
    for (int q = lane; q < SCTA; q += 32)
      if (k0 + q < p.K && isfinite(S_s[q])) m = fminf(m, S_s[q]);
    m = warp_min(m);
    float eta = 0.f, eta_imp = 0.f, sq = 0.f, nf = 0.f;
    for (int q = lane; q < SCTA; q += 32) {
      const int kq = k0 + q;
      const bool fin = kq < p.K && isfinite(S_s[q]);
      const float e = (fin && isfinite(m)) ? expf(-(S_s[q] - m) * p.inv_lambda) : 0.0f;
      e_s[q] = e;
      eta += e;
      eta_imp += (kq < p.n_imp) ? e : 0.0f;
      sq += e * e;
      nf += fin ? 1.0f : 0.0f;
    }
    eta = warp_sum(eta); eta_imp = warp_sum(eta_imp); sq = warp_sum(sq); nf = warp_sum(nf);
    if (lane == 0) {
      rec[0] = m; rec[1] = eta; rec[2] = eta_imp; rec[3] = sq; rec[4] = nf;
      rec[5] = 0.f; rec[6] = 0.f; rec[7] = 0.f;
    }
  }
  __syncthreads();
  {
    const float *ef = reinterpret_cast<const float *>(eps_s);
    for (int o = tid; o < 2 * T; o += NT) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < SCTA; ++q) acc = fmaf(e_s[q], ef[(size_t)q * T * 2 + o], acc);
      rec[8 + o] = acc;
    }
  }

  // ---- phase 5 (cooperative launch): grid barrier, then a slice of the merge per CTA ----
  if (p.coop) {
    if (grid_barrier(p, gen0)) coop_tail<NT, SCTA>(p, S_s, k0);
    return;
  }

  // ---- phase 5: merge by the last CTA of each group; a second level when there are several groups ----
  __shared__ bool am_last;
  __shared__ __align__(8) uint64_t mbar;
  const int nC = gridDim.x;
  const int G = p.group;
  const int g = blockIdx.x / G;
  const int nG = (nC + G - 1) / G;
  const int g0 = g * G, gn = min(G, nC - g0);
  __threadfence();
  __syncthreads();
  if (tid == 0) am_last = (atomicAdd(p.counters + 1 + g, 1u) == (unsigned)(gn - 1));
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // every phase-1..4 buffer is dead now: stage the merge through them
  float *stage = reinterpret_cast<float *>(smem + L.eps);
  const int cap = p.stage_floats;
  if (tid == 0) mbar_init(&mbar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int PL = partial_len(T);
  if (nG == 1) {
    merge_records<NT>(p, p.partials, gn, nullptr, stage, cap, &mbar, phase);
    if (tid == 0) p.counters[1] = 0u;  // ready for the next launch
    return;
  }
  if (!merge_records<NT>(p, p.partials + (size_t)g0 * PL, gn, p.group_rec + (size_t)g * PL, stage, cap, &mbar,
                         phase)) {
    if (tid == 0) p.counters[1 + g] = 0u;
    return;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    p.counters[1 + g] = 0u;
    am_last = (atomicAdd(p.counters, 1u) == (unsigned)(nG - 1));
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  merge_records<NT>(p, p.group_rec, nG, nullptr, stage, cap, &mbar, phase);
  if (tid == 0) p.counters[0] = 0u;  // ready for the next launch
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

struct DeviceInfo {
  int sms = 0;
  size_t smem_optin = 0, smem_per_sm = 0;
};

cudaError_t device_info(DeviceInfo &out) {
  static DeviceInfo cache[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (cache[dev].sms == 0) {
    int sms = 0, optin = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
      return e;
    cache[dev].smem_optin = (size_t)optin;
    cache[dev].smem_per_sm = (size_t)per_sm;
    cache[dev].sms = sms;
  }
  out = cache[dev];
  return cudaSuccess;
}

template <int H, int NW, int SPW, int ACT>
cudaError_t launch_tile(const IterParams &p, int group, cudaStream_t s) {
  const SmemLayout L = fp32_layout(p.T, H, NW, SPW);
  auto kern = iterate_fp32_kernel<H, NW, SPW, ACT>;
  DeviceInfo di;
  cudaError_t e = device_info(di);
  if (e != cudaSuccess) return e;
  const int nC = (p.K + NW * SPW - 1) / (NW * SPW);
  // Shared memory for staging one merge (all of a group's records) when the
  // occupancy the grid needs still fits; otherwise the merge works in chunks.
  const int per_merge = nC <= group ? nC : group;
  const size_t PLb = sizeof(float) * (size_t)partial_len(p.T);
  const size_t want = L.eps + sizeof(float) * (size_t)((per_merge + 3) & ~3) + PLb * per_merge;
  const int ctas_per_sm = (nC + di.sms - 1) / di.sms;
  size_t budget = di.smem_per_sm / (size_t)ctas_per_sm;
  budget = budget > 1024 ? budget - 1024 : 0;  // per-CTA reservation
  if (budget > di.smem_optin) budget = di.smem_optin;
  size_t smem = L.total;
  if (want > smem && want <= budget) smem = want;
  static size_t configured[64] = {};  // largest dynamic shared memory size set so far, per device
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (smem > configured[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = smem;
  }
  IterParams q = p;
  q.group = group;
  q.stage_floats = (int)((smem - L.eps) / sizeof(float));
  // Cooperative launch when every CTA can be resident at once and the U' slices
  // fit the tail's per-CTA bound; otherwise the last-CTA merge tree.
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
  q.coop = (per_sm * di.sms >= nC) && (nC <= 2 * NW * 32) && ((T2 + nC - 1) / nC <= 8) && p.grid_bar != nullptr;
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

constexpr int kMinWarps = 4;         // smallest CTA the picker returns
constexpr int kSingleLevel = 256;    // at most this many CTA records: one merge level
constexpr int kGroup = 128;          // otherwise: CTAs per first-level merge group

int group_for(int nC) { return nC <= kSingleLevel ? nC : kGroup; }

}  // namespace

Fp32Tile fp32_pick_tile(int K, int T, int H, size_t smem_limit) {
  DeviceInfo di;
  const int sms = device_info(di) == cudaSuccess && di.sms > 0 ? di.sms : 148;
  if (H == 32) {
    // Two samples per warp; spread the samples evenly over the SMs, at most 8
    // warps (the register file holds one such CTA per SM).
    const int want = (K + 2 * sms - 1) / (2 * sms);
    int nw = want <= 2 ? 2 : (want <= 4 ? 4 : (want <= 7 ? 7 : 8));
    while (nw > 2 && fp32_layout(T, H, nw, 2).total > smem_limit) nw = nw > 4 ? 4 : 2;
    const int nC = (K + 2 * nw - 1) / (2 * nw);
    return {nw, group_for(nC), 2};
  }
  // One warp per sample.  Large CTAs give few partial records (a short merge).
  int nw = K >= 2048 ? 16 : (K >= 1024 ? 8 : 4);
  while (nw > kMinWarps && fp32_layout(T, H, nw, 1).total > smem_limit) nw = nw > 8 ? 8 : nw / 2;
  const int nC = (K + nw - 1) / nw;
  return {nw, group_for(nC), 1};
}

Fp32Scratch fp32_scratch(int K, int T_max, int H) {
  (void)H;
  const size_t PL = (size_t)partial_len(T_max);
  const size_t nC = (size_t)(K + kMinWarps - 1) / kMinWarps;
  const size_t G = (size_t)group_for((int)nC);
  const size_t nG = (nC + G - 1) / G;
  return {PL * nC, PL * nG, nC > nG ? nC : nG, 1 + nG + 2};  // + grid barrier (arrivals, generation)
}

size_t fp32_smem_bytes(int T, int H, Fp32Tile t) { return fp32_layout(T, H, t.nwarps, t.spw).total; }

int fp32_num_ctas(int K, Fp32Tile t) { return (K + t.nwarps * t.spw - 1) / (t.nwarps * t.spw); }

cudaError_t fp32_launch_iterate(const IterParams &p, Fp32Tile tile, cudaStream_t s) {
#define ITMPC_TILE(HH, WW, SS)                                                                          \
  if (p.H == HH && tile.nwarps == WW && tile.spw == SS)                                                 \
    return p.activation == 1 ? launch_tile<HH, WW, SS, 1>(p, tile.group, s)                             \
                             : launch_tile<HH, WW, SS, 0>(p, tile.group, s);
  ITMPC_TILE(32, 2, 2)
  ITMPC_TILE(32, 4, 2)
  ITMPC_TILE(32, 7, 2)
  ITMPC_TILE(32, 8, 2)
  ITMPC_TILE(64, 4, 1)
  ITMPC_TILE(64, 8, 1)
  ITMPC_TILE(64, 16, 1)
  ITMPC_TILE(128, 4, 1)
  ITMPC_TILE(128, 8, 1)
  ITMPC_TILE(128, 16, 1)
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
