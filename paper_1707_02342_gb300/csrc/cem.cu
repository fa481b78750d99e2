// cem.cu -- cross-entropy weights (Alg. 3) and the cross-entropy control update on the GPU.
//
// Alg. 3: zeta = round(K (1 - delta)), Z = the zeta-th smallest cost, uniform weights on
// the elite set {k : S_k <= Z} (1/|E|, |E| = zeta without ties; the elite set of the
// method's own definition -- the printed strict inequality would give weights summing to
// (zeta - 1)/zeta), then the same control law U'_t = sum_k w_k v_{k,t}: the un-weighted
// mean of the elite controls.
//   cem_select_kernel  one CTA: the zeta-th smallest finite cost by a 4-pass radix select
//                      over order-preserving 32-bit keys (256-bin shared histograms,
//                      one 8-bit digit per pass), the elite count, the weights;
//   cem_update_kernel  one CTA per step t: the mean of the elite samples' v_{k,t}, the
//                      noise drawn again from its Philox counter; fixed-order reduction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"

namespace itmpc {

namespace {

constexpr int kSelThreads = 1024;
constexpr int kUpdThreads = 256;

// Monotone map of finite floats to unsigned keys (a < b  <=>  key(a) < key(b)).
__device__ __forceinline__ uint32_t fkey(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_to_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Sum over the CTA, identical in every thread (fixed order over the warps).
__device__ float block_sum(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.0f;
  for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];  // same order in every thread
  return s;
}

constexpr int kKeysInSmem = 11264;  // up to this many keys are staged in shared memory (44 KB + 1.2 KB static)
constexpr uint32_t kNonFinite = 0xFFFFFFFFu;  // above every finite key

__global__ void __launch_bounds__(kSelThreads) cem_select_kernel(int K, int zeta0, const float *__restrict__ S,
                                                                 float *w, float *scal, int *status) {
  __shared__ unsigned int hist[256];
  __shared__ float red[32];
  __shared__ uint32_t prefix_s;
  __shared__ int rank_s;
  extern __shared__ uint32_t keys_s[];  // K keys when K <= kKeysInSmem
  const int tid = threadIdx.x, lane = tid & 31;
  const bool staged = K <= kKeysInSmem;
  auto key_at = [&](int k) -> uint32_t {
    if (staged) return keys_s[k];
    const float v = S[k];
    return isfinite(v) ? fkey(v) : kNonFinite;
  };
  // finite costs and the clamped rank
  float nf = 0.0f;
  for (int k = tid; k < K; k += kSelThreads) {
    const float v = S[k];
    const bool fin = isfinite(v);
    nf += fin ? 1.0f : 0.0f;
    if (staged) keys_s[k] = fin ? fkey(v) : kNonFinite;
  }
  const int n_fin = (int)block_sum(nf, red);  // (its barriers also publish keys_s)
  if (n_fin == 0) {
    for (int k = tid; k < K; k += kSelThreads) w[k] = 0.0f;
    if (tid == 0) {
      scal[0] = NAN;
      scal[1] = 0.0f;
      *status = -3;  // every cost non-finite: the caller's U is kept
    }
    return;
  }
  int rank = min(max(zeta0, 1), n_fin);  // 1-based rank of Z among the finite costs
  uint32_t prefix = 0u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t hi_mask = pass == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (int i = tid; i < 256; i += kSelThreads) hist[i] = 0u;
    __syncthreads();
    for (int k = tid; k < K; k += kSelThreads) {
      const uint32_t key = key_at(k);
      if (key == kNonFinite) continue;
      if ((key & hi_mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    if (tid < 32) {
      // the digit holding rank r: lane l owns bins 8 l .. 8 l + 7; a warp scan of the lane
      // totals finds the lane, which then walks its eight bins
      int cnt[8], tot = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        cnt[b] = (int)hist[8 * lane + b];
        tot += cnt[b];
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += n;
      }
      const unsigned hit = __ballot_sync(FULL_MASK, incl >= rank);
      const int owner = hit ? __ffs(hit) - 1 : 31;
      if (lane == owner) {
        int r = rank - (incl - tot), d = 8 * lane;
#pragma unroll 1
        for (int b = 0; b < 7 && cnt[b] < r; ++b) {
          r -= cnt[b];
          ++d;
        }
        prefix_s = prefix | ((uint32_t)d << shift);
        rank_s = r;
      }
    }
    __syncthreads();
    prefix = prefix_s;
    rank = rank_s;
  }
  const uint32_t zkey = prefix;
  float ne = 0.0f;
  for (int k = tid; k < K; k += kSelThreads) ne += key_at(k) <= zkey ? 1.0f : 0.0f;
  const float m = block_sum(ne, red);
  const float inv = 1.0f / m;
  for (int k = tid; k < K; k += kSelThreads) w[k] = key_at(k) <= zkey ? inv : 0.0f;
  if (tid == 0) {
    scal[0] = key_to_float(zkey);
    scal[1] = m;
  }
}

__global__ void __launch_bounds__(kUpdThreads) cem_update_kernel(const IterParams p, const float *__restrict__ w,
                                                                 const float *__restrict__ scal) {
  __shared__ float red[32];
  const int t = blockIdx.x;
  const float m = scal[1];
  const float u0 = __ldg(p.U + 2 * t), u1 = __ldg(p.U + 2 * t + 1);
  if (!(m > 0.0f)) {  // no finite cost: U unchanged
    if (threadIdx.x == 0) {
      p.U_out[2 * t] = u0;
      p.U_out[2 * t + 1] = u1;
    }
    return;
  }
  float a0 = 0.0f, a1 = 0.0f;
  for (int k = threadIdx.x; k < p.K; k += kUpdThreads) {
    if (w[k] == 0.0f) continue;
    const float2 e = noise_at(p, (uint32_t)k, (uint32_t)t);
    const bool imp = k < p.n_imp;
    a0 += imp ? u0 + e.x : e.x;
    a1 += imp ? u1 + e.y : e.y;
  }
  const float s0 = block_sum(a0, red);
  const float s1 = block_sum(a1, red);
  if (threadIdx.x == 0) {
    p.U_out[2 * t] = s0 / m;
    p.U_out[2 * t + 1] = s1 / m;
  }
}

}  // namespace

cudaError_t cem_launch(const IterParams &p, int zeta0, const float *S, float *w, float *scal, cudaStream_t s) {
  const size_t smem = p.K <= kKeysInSmem ? sizeof(uint32_t) * (size_t)p.K : 0;
  cem_select_kernel<<<1, kSelThreads, smem, s>>>(p.K, zeta0, S, w, scal, p.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cem_update_kernel<<<p.T, kUpdThreads, 0, s>>>(p, w, scal);
  return cudaGetLastError();
}

}  // namespace itmpc
