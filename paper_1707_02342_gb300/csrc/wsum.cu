// wsum.cu -- the control law of Sec. III-D from materialised noise:
//   U'_t = sum_k w_k v_{k,t} = U_t sum_{k importance} w_k + sum_k w_k eps_{k,t}
// for a caller that holds eps (K x T x 2, row k contiguous) in device memory.  This is the
// HBM-bound form of the update (K T 8 bytes streamed once), beside the fused iteration,
// which never writes eps.
//   wsum_partial4_kernel a CTA streams a contiguous slab of rows; thread (row group ry,
//                        column c) accumulates w_k eps over its rows with 16-byte loads
//                        coalesced along t (two steps per load, even T and a 16-byte aligned
//                        eps); the row groups are summed in shared memory in a fixed order;
//                        one partial record per CTA (2T sums and the slab's importance-weight
//                        sum);
//   wsum_partial_kernel  the same with 8-byte loads (one step), for odd T;
//   wsum_final_kernel    sums the records in a fixed order (32 interleaved record groups,
//                        then group order) and adds U_t times the importance weight.
#include <cuda_runtime.h>
#include <stdint.h>

#include "itmpc_device.cuh"

namespace itmpc {

namespace {

constexpr int kWsThreads = 256;
constexpr int kWsCtasPerSm = 4;

// Record stride in floats: 2T sums, the slab's importance-weight sum, padded to a multiple of
// 4 floats so that every record starts on a 16-byte boundary.
__host__ __device__ __forceinline__ int ws_stride(int T) { return (2 * T + 1 + 3) & ~3; }

__global__ void __launch_bounds__(kWsThreads) wsum_partial_kernel(int K, int T, int n_imp, int rows_per_cta,
                                                                 const float2 *__restrict__ eps,
                                                                 const float *__restrict__ w, float *part) {
  extern __shared__ float2 red[];  // kWsThreads float2
  const int TC = T < kWsThreads ? T : kWsThreads;  // step columns handled at once
  const int R = kWsThreads / TC;                     // row groups
  const int tid = threadIdx.x, c = tid % TC, ry = tid / TC;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(K, r0 + rows_per_cta);
  const int PS = ws_stride(T);
  float *rec = part + (size_t)blockIdx.x * PS;
  {
    __shared__ float wred[kWsThreads / 32];
    float wi = 0.0f;
    for (int k = r0 + tid; k < min(r1, n_imp); k += kWsThreads) wi += __ldg(w + k);
    wi = warp_sum(wi);
    if ((tid & 31) == 0) wred[tid >> 5] = wi;
    __syncthreads();
    if (tid == 0) {
      float sw = 0.0f;
      for (int g = 0; g < kWsThreads / 32; ++g) sw += wred[g];
      rec[2 * T] = sw;
    }
  }
  for (int cb = 0; cb < T; cb += TC) {
    const int t = cb + c;
    float2 acc = make_float2(0.0f, 0.0f);
    if (ry < R && t < T) {
#pragma unroll 8
      for (int k = r0 + ry; k < r1; k += R) {
        const float wk = __ldg(w + k);
        const float2 e = __ldcs(eps + (size_t)k * T + t);  // streamed once: evict first
        acc.x = fmaf(wk, e.x, acc.x);
        acc.y = fmaf(wk, e.y, acc.y);
      }
    }
    red[tid] = acc;
    __syncthreads();
    if (ry == 0 && t < T) {
      float2 s = red[c];
      for (int g = 1; g < R; ++g) {
        s.x += red[g * TC + c].x;
        s.y += red[g * TC + c].y;
      }
      reinterpret_cast<float2 *>(rec)[t] = s;
    }
    __syncthreads();
  }
}

// Even T: rows are 2T floats = T/2 float4 (16-byte aligned rows), so each thread streams
// 16-byte loads; thread (row group ry, column c) covers steps 2c and 2c + 1.
__global__ void __launch_bounds__(kWsThreads) wsum_partial4_kernel(int K, int T, int n_imp, int rows_per_cta,
                                                                  const float4 *__restrict__ eps,
                                                                  const float *__restrict__ w, float *part) {
  __shared__ float4 red4[kWsThreads];
  __shared__ float wred[kWsThreads / 32];
  const int W4 = T / 2;                                  // float4 per row
  const int TC = W4 < kWsThreads ? W4 : kWsThreads;     // columns handled at once
  const int R = kWsThreads / TC;                         // row groups
  const int tid = threadIdx.x, c = tid % TC, ry = tid / TC;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(K, r0 + rows_per_cta);
  const int PS = ws_stride(T);
  float *rec = part + (size_t)blockIdx.x * PS;
  float wi = 0.0f;
  for (int k = r0 + tid; k < min(r1, n_imp); k += kWsThreads) wi += __ldg(w + k);
  wi = warp_sum(wi);
  if ((tid & 31) == 0) wred[tid >> 5] = wi;
  __syncthreads();
  if (tid == 0) {
    float sw = 0.0f;
    for (int g = 0; g < kWsThreads / 32; ++g) sw += wred[g];
    rec[2 * T] = sw;
  }
  for (int cb = 0; cb < W4; cb += TC) {
    const int col = cb + c;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (ry < R && col < W4) {
      const float4 *p = eps + (size_t)(r0 + ry) * W4 + col;
      const size_t stride = (size_t)R * W4;
#pragma unroll 8
      for (int k = r0 + ry; k < r1; k += R, p += stride) {
        const float wk = __ldg(w + k);
        const float4 e = __ldcs(p);  // streamed once: evict first
        acc.x = fmaf(wk, e.x, acc.x);
        acc.y = fmaf(wk, e.y, acc.y);
        acc.z = fmaf(wk, e.z, acc.z);
        acc.w = fmaf(wk, e.w, acc.w);
      }
    }
    red4[tid] = acc;
    __syncthreads();
    if (ry == 0 && col < W4) {
      float4 s = red4[c];
      for (int g = 1; g < R; ++g) {
        const float4 o = red4[g * TC + c];
        s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
      }
      reinterpret_cast<float4 *>(rec)[col] = s;  // records start on 16-byte boundaries
    }
    __syncthreads();
  }
}

// Thread (record group g, element column c): group g sums records g, g + 32, g + 64, ... of
// its column; the 32 group sums are then added in group order (a fixed order for any launch).
// 8 columns per CTA keep 2T/8 CTAs busy on the short reduction.
constexpr int kWfCols = 8;
constexpr int kWfGroups = kWsThreads / kWfCols;

__global__ void __launch_bounds__(kWsThreads) wsum_final_kernel(int n_cta, int T, const float *__restrict__ part,
                                                               const float *__restrict__ U, float *U_out) {
  __shared__ float red[kWfGroups][kWfCols + 1];
  __shared__ float redw[kWfGroups][kWfCols + 1];
  const int c = threadIdx.x % kWfCols, g = threadIdx.x / kWfCols;
  const int e = blockIdx.x * kWfCols + c;
  const int PS = ws_stride(T);
  float s = 0.0f, w_imp = 0.0f;
  if (e < 2 * T) {
#pragma unroll 8
    for (int b = g; b < n_cta; b += kWfGroups) {
      s += part[(size_t)b * PS + e];
      w_imp += part[(size_t)b * PS + 2 * T];
    }
  }
  red[g][c] = s;
  redw[g][c] = w_imp;
  __syncthreads();
  if (g == 0 && e < 2 * T) {
    float st = red[0][c], wt = redw[0][c];
    for (int q = 1; q < kWfGroups; ++q) {
      st += red[q][c];
      wt += redw[q][c];
    }
    U_out[e] = fmaf(__ldg(U + e), wt, st);
  }
}

}  // namespace

size_t wsum_part_floats(int T_max, int sms) { return (size_t)kWsCtasPerSm * sms * (size_t)ws_stride(T_max); }

cudaError_t wsum_launch(int K, int T, int n_imp, const float *eps, const float *w, const float *U, float *U_out,
                        float *part, int sms, cudaStream_t s) {
  const int ctas = kWsCtasPerSm * sms;  // resident CTAs of 256 threads stream contiguous slabs of rows
  const int rows = (K + ctas - 1) / ctas;
  const int n_cta = (K + rows - 1) / rows;
  if (T % 2 == 0 && (reinterpret_cast<uintptr_t>(eps) & 15u) == 0)
    wsum_partial4_kernel<<<n_cta, kWsThreads, 0, s>>>(K, T, n_imp, rows, reinterpret_cast<const float4 *>(eps), w,
                                                      part);
  else
    wsum_partial_kernel<<<n_cta, kWsThreads, sizeof(float2) * kWsThreads, s>>>(
        K, T, n_imp, rows, reinterpret_cast<const float2 *>(eps), w, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wsum_final_kernel<<<(2 * T + kWfCols - 1) / kWfCols, kWsThreads, 0, s>>>(n_cta, T, part, U, U_out);
  return cudaGetLastError();
}

}  // namespace itmpc
