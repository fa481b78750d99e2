// itmpc_merge.cuh -- log-sum-exp merge of per-CTA partial records (Alg. 2 shift
// by the minimum cost, applied per record and then across records).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_sum.cuh"

namespace itmpc {

constexpr int kDevErrNonfinite = -3;  // ITMPC_ERR_NONFINITE
constexpr int kDevErrTimeout = -4;    // ITMPC_ERR_TIMEOUT
constexpr uint32_t kWaitPolls = 1u << 22;  // bounded mbarrier wait: ~0.3 s of 64 ns sleeps

// Pass 1 + 2 of merge_records (whole CTA), from the records in global memory: tot = {rho =
// min rho_c, eta, the importance part of eta, the sum of squares, the finite count}.  The same
// operations in the same order as merge_records' passes 1 + 2, so a CTA that calls it on the
// same records gets the same bits.  tot[1..4] are written by thread 0 after the last barrier:
// the caller synchronises before reading them.  (merge_records keeps its own copy of these
// passes: folding them into a shared function changed the fused kernel's code generation.)
template <int NT>
__device__ void merge_scalars(const IterParams &p, const float *recs, int n, float (*red)[8], float *tot) {
  const int PL = partial_len(p.T);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = NT / 32;
  auto header = [&](int c) -> float4 { return __ldcg(reinterpret_cast<const float4 *>(recs + (size_t)c * PL)); };
  auto nfin = [&](int c) -> float { return __ldcg(recs + (size_t)c * PL + 4); };
  float m = INFINITY;
  for (int c = tid; c < n; c += NT) m = fminf(m, header(c).x);
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
  CSum eta, eta_imp, sq;
  float nf = 0.f;  // a count: exact in FP32 up to 2^24 samples
  for (int c = tid; c < n; c += NT) {
    const float4 h = header(c);
    const float sc = (ok && isfinite(h.x)) ? expf(-(h.x - rho) * p.inv_lambda) : 0.0f;
    eta.add_prod(sc, h.y);
    eta_imp.add_prod(sc, h.z);
    sq.add_prod(__fmul_rn(sc, sc), h.w);
    nf += nfin(c);
  }
  eta = csum_warp(eta);
  eta_imp = csum_warp(eta_imp);
  sq = csum_warp(sq);
  nf = warp_sum(nf);
  __syncthreads();  // tot[0] consumed, scs written
  if (lane == 0) {
    red[warp][0] = eta.s; red[warp][1] = eta.c; red[warp][2] = eta_imp.s; red[warp][3] = eta_imp.c;
    red[warp][4] = sq.s; red[warp][5] = sq.c; red[warp][6] = nf;
  }
  __syncthreads();
  if (tid == 0) {
    CSum a, b, c;
    float d = 0.f;
    for (int w = 0; w < NWARP; ++w) {
      a.add(CSum{red[w][0], red[w][1]});
      b.add(CSum{red[w][2], red[w][3]});
      c.add(CSum{red[w][4], red[w][5]});
      d += red[w][6];
    }
    tot[1] = a.value(); tot[2] = b.value(); tot[3] = c.value(); tot[4] = d;
  }
}

// The weights w_k = exp(-(S_k - rho)/lambda) / eta of samples k = part * 8 NT + ... (every
// nparts-th block of 8 NT), rho and eta from the records as merge_records computes them: the
// merge of one instance spreads its K weights over several CTAs this way.
template <int NT>
__device__ void merge_weights(const IterParams &p, const float *recs, int n, int part, int nparts) {
  __shared__ float red[NT / 32][8];
  __shared__ float tot[5];
  merge_scalars<NT>(p, recs, n, red, tot);
  __syncthreads();  // tot[1] written by thread 0
  const float rho = tot[0];
  const bool ok = isfinite(rho);
  const float inv_eta = ok ? 1.0f / tot[1] : 0.0f;
  const int tid = threadIdx.x;
  for (int kb = part * 8 * NT; kb < p.K; kb += nparts * 8 * NT) {
    float v[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int k = kb + b * NT + tid;
      v[b] = k < p.K ? __ldcg(p.costs + k) : 0.0f;
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int k = kb + b * NT + tid;
      if (k < p.K) p.weights[k] = (ok && isfinite(v[b])) ? expf(-(v[b] - rho) * p.inv_lambda) * inv_eta : 0.0f;
    }
  }
}

// Merge n records (stride PL floats, 16-byte aligned) with the log-sum-exp rule
// of Alg. 2: rho = min rho_c, every record rescaled by exp(-(rho_c - rho)/lambda).
// The whole CTA calls it.  If `out` is non-null the merged record is written
// there; otherwise the final outputs (U', weights, stats) are written.
// Records are staged into shared memory (`stage`, `cap` floats, 16-byte
// aligned) by cp.async.bulk copies completed on `mbar`: all of them with one
// copy when they fit, else chunk by chunk.  The E sums are split over
// (output, record-slice) pairs.  Every sum over records (eta, the importance
// part, the squares, E) is compensated (itmpc_sum.cuh).  Returns false (status
// ITMPC_ERR_TIMEOUT) if a copy did not complete in time.
template <int NT>
__device__ bool merge_records(const IterParams &p, const float *recs, int n, float *out, float *stage, int cap,
                              uint64_t *mbar, uint32_t &phase) {
  const int T = p.T, PL = partial_len(T), T2 = 2 * T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = NT / 32;
  constexpr int MAXO = (2 * ITMPC_MAX_T_DEV + NT - 1) / NT;
  __shared__ float red[NWARP][8];
  __shared__ float tot[5];

  // stage layout: [per-record scale: CH floats, padded to 4][CH records]
  const int CH = max(1, min(n, (cap - 4) / (PL + 1)));
  float *scs = stage;
  float *rs = stage + ((CH + 3) & ~3);
  const bool whole = CH >= n;

  auto copy_chunk = [&](int c0, int cn) -> bool {
    __syncthreads();  // the stage is free (previous chunk consumed, earlier phases done)
    if (tid == 0) {
      fence_proxy_async();
      const uint32_t bytes = (uint32_t)(cn * PL * sizeof(float));
      mbar_expect_tx(mbar, bytes);
      bulk_copy_g2s(rs, recs + (size_t)c0 * PL, bytes, mbar);
    }
    const bool done = mbar_wait_bounded(mbar, phase, kWaitPolls);
    if (__syncthreads_or(!done)) {
      if (tid == 0) *p.status = kDevErrTimeout;
      mbar_wait_bounded(mbar, phase, kWaitPolls);  // let the copy land before the CTA leaves
      return false;
    }
    phase ^= 1u;
    return true;
  };

  // pass 1 + 2: rho and the scalar sums, from the staged records when they all fit
  if (whole && !copy_chunk(0, n)) return false;
  auto header = [&](int c) -> float4 {
    return whole ? *reinterpret_cast<const float4 *>(rs + (size_t)c * PL)
                 : __ldcg(reinterpret_cast<const float4 *>(recs + (size_t)c * PL));
  };
  auto nfin = [&](int c) -> float { return whole ? rs[(size_t)c * PL + 4] : __ldcg(recs + (size_t)c * PL + 4); };
  float m = INFINITY;
  for (int c = tid; c < n; c += NT) m = fminf(m, header(c).x);
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
  CSum eta, eta_imp, sq;
  float nf = 0.f;  // a count: exact in FP32 up to 2^24 samples
  for (int c = tid; c < n; c += NT) {
    const float4 h = header(c);
    const float sc = (ok && isfinite(h.x)) ? expf(-(h.x - rho) * p.inv_lambda) : 0.0f;
    if (whole) scs[c] = sc;
    eta.add_prod(sc, h.y);
    eta_imp.add_prod(sc, h.z);
    sq.add_prod(__fmul_rn(sc, sc), h.w);
    nf += nfin(c);
  }
  eta = csum_warp(eta);
  eta_imp = csum_warp(eta_imp);
  sq = csum_warp(sq);
  nf = warp_sum(nf);
  __syncthreads();  // tot[0] consumed, scs written
  if (lane == 0) {
    red[warp][0] = eta.s; red[warp][1] = eta.c; red[warp][2] = eta_imp.s; red[warp][3] = eta_imp.c;
    red[warp][4] = sq.s; red[warp][5] = sq.c; red[warp][6] = nf;
  }
  __syncthreads();
  if (tid == 0) {
    CSum a, b, c;
    float d = 0.f;
    for (int w = 0; w < NWARP; ++w) {
      a.add(CSum{red[w][0], red[w][1]});
      b.add(CSum{red[w][2], red[w][3]});
      c.add(CSum{red[w][4], red[w][5]});
      d += red[w][6];
    }
    tot[1] = a.value(); tot[2] = b.value(); tot[3] = c.value(); tot[4] = d;
  }

  // pass 3: E sums.  Thread -> (output o, record slice r) when 2T <= NT.
  const int S = T2 <= NT ? NT / T2 : 1;
  const int r = T2 <= NT ? tid / T2 : 0;
  const bool active = T2 <= NT ? (tid < S * T2) : true;
  CSum acc[MAXO];
  for (int c0 = 0; c0 < n; c0 += CH) {
    const int cn = min(CH, n - c0);
    if (!whole) {
      if (!copy_chunk(c0, cn)) return false;
      for (int c = tid; c < cn; c += NT) {
        const float rc = rs[(size_t)c * PL];
        scs[c] = (ok && isfinite(rc)) ? expf(-(rc - rho) * p.inv_lambda) : 0.0f;
      }
      __syncthreads();
    }
    if (ok && active) {
#pragma unroll
      for (int j = 0; j < MAXO; ++j) {
        const int o = T2 <= NT ? tid % T2 : tid + j * NT;
        if ((j == 0 || T2 > NT) && o < T2) {
          CSum a0, a1;
          int c = r;
          for (; c + S < cn; c += 2 * S) {
            a0.add_prod(scs[c], rs[(size_t)c * PL + 8 + o]);
            a1.add_prod(scs[c + S], rs[(size_t)(c + S) * PL + 8 + o]);
          }
          if (c < cn) a0.add_prod(scs[c], rs[(size_t)c * PL + 8 + o]);
          acc[j].add(a0);
          acc[j].add(a1);
        }
      }
    }
  }
  // combine the record slices through shared memory (reusing the stage): (s, c) pairs
  __syncthreads();
  float *part = stage;
  if (T2 <= NT && active) {
    part[2 * (r * T2 + (tid % T2))] = acc[0].s;
    part[2 * (r * T2 + (tid % T2)) + 1] = acc[0].c;
  }
  __syncthreads();
  const float eta_t = tot[1], eta_imp_t = tot[2], sq_t = tot[3], nf_t = tot[4];
  const float inv_eta = ok ? 1.0f / eta_t : 0.0f;
  const float imp_frac = eta_imp_t * inv_eta;
#pragma unroll
  for (int j = 0; j < MAXO; ++j) {
    const int o = tid + j * NT;
    if (o < T2) {
      float E;
      if (T2 <= NT) {
        CSum Ec;
        for (int q = 0; q < S; ++q) Ec.add(CSum{part[2 * (q * T2 + o)], part[2 * (q * T2 + o) + 1]});
        E = Ec.value();
      } else {
        E = acc[j].value();
      }
      if (out) {
        out[8 + o] = ok ? E : 0.0f;
      } else {
        const float u = p.U[o];
        p.U_out[o] = ok ? u * imp_frac + E * inv_eta : u;
      }
    }
  }
  if (out) {
    if (tid == 0) {
      out[0] = rho; out[1] = eta_t; out[2] = eta_imp_t; out[3] = sq_t; out[4] = nf_t;
      out[5] = 0.f; out[6] = 0.f; out[7] = 0.f;
    }
    return true;
  }
  if (p.weights && p.weights_inline) {
    // all loads of a batch are issued before its stores
    for (int kb = 0; kb < p.K; kb += 8 * NT) {
      float v[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int k = kb + b * NT + tid;
        v[b] = k < p.K ? __ldcg(p.costs + k) : 0.0f;
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int k = kb + b * NT + tid;
        if (k < p.K) p.weights[k] = (ok && isfinite(v[b])) ? expf(-(v[b] - rho) * p.inv_lambda) * inv_eta : 0.0f;
      }
    }
  }
  if (tid == 0) {
    p.stats[0] = rho;
    p.stats[1] = eta_t;
    p.stats[2] = ok ? eta_t * eta_t / sq_t : 0.0f;
    p.stats[3] = ok ? rho - p.lambda * logf(eta_t / (float)p.K) : INFINITY;
    p.stats[4] = nf_t;
    p.stats[5] = 0.f; p.stats[6] = 0.f; p.stats[7] = 0.f;
    if (!ok) *p.status = kDevErrNonfinite;
  }
  return true;
}

}  // namespace itmpc
