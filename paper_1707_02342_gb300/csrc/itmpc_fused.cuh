// itmpc_fused.cuh -- the end of a fused iteration kernel, shared by the kernels of
// the network widths: the CTA's partial record (Alg. 2 over the CTA's samples:
// rho_c = min S, eta_c = sum e, the importance part, sum e^2, the finite count and
// E_c = sum e eps with e = exp(-(S - rho_c)/lambda), every sum compensated) and the
// merge of the records into U' (Sec. III-D), the weights and the diagnostics:
// either a bounded grid barrier followed by a slice of the merge in every CTA (a
// cooperative launch, every CTA resident), or the last-arriving CTA of each group
// of CTAs merging the group's records and the last group merger finishing.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_merge.cuh"
#include "itmpc_sum.cuh"

namespace itmpc {

// ---- cooperative tail: a grid barrier, then every CTA merges a slice ----
static __device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr uint32_t kBarrierPolls = 1u << 24;  // bounded wait: ~1 s of 64 ns sleeps

static __device__ __forceinline__ unsigned atom_add_release_u32(unsigned *p, unsigned v) {
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
static __device__ bool grid_barrier(const IterParams &p, unsigned gen0) {
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
  __shared__ float red[NWARP][2 * (5 + MAXS)];
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
  // pass 2: scalar sums and this CTA's E slice (compensated: itmpc_sum.cuh)
  CSum acc[5 + MAXS];
#pragma unroll
  for (int j = 0; j < MAXR; ++j) {
    const float4 h = hdr[j];
    const float sc = (ok && isfinite(h.x)) ? expf(-(h.x - rho) * p.inv_lambda) : 0.0f;
    acc[0].add_prod(sc, h.y);
    acc[1].add_prod(sc, h.z);
    acc[2].add_prod(__fmul_rn(sc, sc), h.w);
    acc[3].s += nfr[j];  // a count: exact
#pragma unroll
    for (int q = 0; q < MAXS; ++q)
      if (q < on) acc[5 + q].add_prod(sc, evr[j][q]);
  }
  __syncthreads();  // tot[0] consumed
  // only the sums this CTA uses: eta, the importance part, the squares, the count (4 is unused)
  // and its `on` outputs of U'
#pragma unroll
  for (int q = 0; q < 5 + MAXS; ++q) {
    if (q == 4 || q >= 5 + on) continue;  // block-uniform
    const CSum v = q == 3 ? CSum{warp_sum(acc[3].s), 0.f} : csum_warp(acc[q]);
    if (lane == 0) {
      red[warp][2 * q] = v.s;
      red[warp][2 * q + 1] = v.c;
    }
  }
  __syncthreads();
  if (tid < 5 + on && tid != 4) {
    CSum a;
    for (int w = 0; w < NWARP; ++w) a.add(CSum{red[w][2 * tid], red[w][2 * tid + 1]});
    tot[tid] = a.value();
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

// Phase 4 + 5 of a fused iteration, called by every thread of the CTA after the
// costs of its SCTA samples are in S_s (samples k0 .. k0 + SCTA - 1):
//   eps        the CTA's noise: sample q's eps[t][i] at
//              eps[(q / EG) * eps_stride + (q % EG) * 2 T + 2 t + i] (groups of EG samples
//              with contiguous rows, eps_stride floats apart);
//   e_s        SCTA floats of shared scratch;
//   gen0       the grid-barrier generation read before this launch's barrier;
//   stage      shared memory for the merge (p.stage_floats floats; the rollout's buffers).
template <int NT, int SCTA, int EG = 1>
__device__ void record_and_merge(const IterParams &p, const float *S_s, float *e_s, const float *eps,
                                 size_t eps_stride, int k0, unsigned gen0, float *stage) {
  const int T = p.T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- phase 4: this CTA's partial record ----
  float *rec = p.partials + (size_t)blockIdx.x * partial_len(T);
  if (warp == 0) {
    float m = INFINITY;
    for (int q = lane; q < SCTA; q += 32)
      if (k0 + q < p.K && isfinite(S_s[q])) m = fminf(m, S_s[q]);
    m = warp_min(m);
    CSum eta, eta_imp, sq;
    float nf = 0.f;
    for (int q = lane; q < SCTA; q += 32) {
      const int kq = k0 + q;
      const bool fin = kq < p.K && isfinite(S_s[q]);
      const float e = (fin && isfinite(m)) ? expf(-(S_s[q] - m) * p.inv_lambda) : 0.0f;
      e_s[q] = e;
      eta.add(e);
      eta_imp.add(((long long)p.k_base + kq < p.n_imp) ? e : 0.0f);
      sq.add_prod(e, e);
      nf += fin ? 1.0f : 0.0f;
    }
    eta = csum_warp(eta); eta_imp = csum_warp(eta_imp); sq = csum_warp(sq); nf = warp_sum(nf);
    if (lane == 0) {
      rec[0] = m; rec[1] = eta.value(); rec[2] = eta_imp.value(); rec[3] = sq.value(); rec[4] = nf;
      rec[5] = 0.f; rec[6] = 0.f; rec[7] = 0.f;
    }
  }
  __syncthreads();
  for (int o = tid; o < 2 * T; o += NT) {
    CSum acc;
#pragma unroll
    for (int q = 0; q < SCTA; ++q) acc.add_prod(e_s[q], eps[(size_t)(q / EG) * eps_stride + (q % EG) * 2 * T + o]);
    rec[8 + o] = acc.value();
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
  // every buffer of the rollout is dead now: stage the merge through them
  const int cap = p.stage_floats;
  if (tid == 0) mbar_init(&mbar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int PL = partial_len(T);
  if (nG == 1) {
    merge_records<NT>(p, p.partials, gn, p.rec_out, stage, cap, &mbar, phase);
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
  merge_records<NT>(p, p.group_rec, nG, p.rec_out, stage, cap, &mbar, phase);
  if (tid == 0) p.counters[0] = 0u;  // ready for the next launch
}

struct DeviceInfo {
  int sms = 0;
  size_t smem_optin = 0, smem_per_sm = 0;
};

inline cudaError_t device_info(DeviceInfo &out) {
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

}  // namespace itmpc
