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
// The sums are compensated (itmpc_sum.cuh) at block granularity: a thread adds
// kWsBlock rows with plain FMAs (their loads in flight together) and folds each block
// sum into a (sum, correction) pair with Neumaier's step, so the rounding error grows
// with the block length, not with the thousands of rows a thread streams; partial
// sums are merged as pairs.  A compensated step per element would make this
// HBM-bound kernel instruction-bound.
#include <cuda_runtime.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_sum.cuh"

namespace itmpc {

namespace {

constexpr int kWsThreads = 256;
constexpr int kWsBlock = 8;  // rows per plain-FMA block of a thread's compensated sum
constexpr int kWsCtasPerSm = 4;

// Record stride in floats: 2T sums, the slab's importance-weight sum, padded to a multiple of
// 4 floats so that every record starts on a 16-byte boundary.
__host__ __device__ __forceinline__ int ws_stride(int T) { return (2 * T + 1 + 3) & ~3; }

__global__ void __launch_bounds__(kWsThreads, kWsCtasPerSm) wsum_partial_kernel(int K, int T, int n_imp, int rows_per_cta,
                                                                 const float2 *__restrict__ eps,
                                                                 const float *__restrict__ w, float *part) {
  extern __shared__ float2 red[];  // 2 kWsThreads float2: (sum, correction) of x and y
  const int TC = T < kWsThreads ? T : kWsThreads;  // step columns handled at once
  const int R = kWsThreads / TC;                     // row groups
  const int tid = threadIdx.x, c = tid % TC, ry = tid / TC;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(K, r0 + rows_per_cta);
  const int PS = ws_stride(T);
  float *rec = part + (size_t)blockIdx.x * PS;
  {
    __shared__ float2 wred[kWsThreads / 32];
    CSum wi;
    for (int k = r0 + tid; k < min(r1, n_imp); k += kWsThreads) wi.add(__ldg(w + k));
    wi = csum_warp(wi);
    if ((tid & 31) == 0) wred[tid >> 5] = make_float2(wi.s, wi.c);
    __syncthreads();
    if (tid == 0) {
      CSum sw;
      for (int g = 0; g < kWsThreads / 32; ++g) sw.add(CSum{wred[g].x, wred[g].y});
      rec[2 * T] = sw.value();
    }
  }
  for (int cb = 0; cb < T; cb += TC) {
    const int t = cb + c;
    CSum ax, ay;
    if (ry < R && t < T) {
      // blocks of kWsBlock rows: plain FMAs (loads in flight), then one compensated step per block
      for (int kb = r0 + ry; kb < r1; kb += kWsBlock * R) {
        float2 ev[kWsBlock];
        float wv[kWsBlock];
#pragma unroll
        for (int u = 0; u < kWsBlock; ++u) {  // every load of the block in flight
          const int k = kb + u * R;
          wv[u] = k < r1 ? __ldg(w + k) : 0.0f;
          ev[u] = k < r1 ? __ldcs(eps + (size_t)k * T + t) : make_float2(0.0f, 0.0f);  // streamed once
        }
        float2 blk = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < kWsBlock; ++u) {
          blk.x = fmaf(wv[u], ev[u].x, blk.x);
          blk.y = fmaf(wv[u], ev[u].y, blk.y);
        }
        ax.add(blk.x);
        ay.add(blk.y);
      }
    }
    red[2 * tid] = make_float2(ax.s, ax.c);
    red[2 * tid + 1] = make_float2(ay.s, ay.c);
    __syncthreads();
    if (ry == 0 && t < T) {
      CSum sx, sy;
      for (int g = 0; g < R; ++g) {
        const float2 qx = red[2 * (g * TC + c)], qy = red[2 * (g * TC + c) + 1];
        sx.add(CSum{qx.x, qx.y});
        sy.add(CSum{qy.x, qy.y});
      }
      reinterpret_cast<float2 *>(rec)[t] = make_float2(sx.value(), sy.value());
    }
    __syncthreads();
  }
}

// Even T: rows are 2T floats = T/2 float4 (16-byte aligned rows), so each thread streams
// 16-byte loads; thread (row group ry, column c) covers steps 2c and 2c + 1.
__global__ void __launch_bounds__(kWsThreads, kWsCtasPerSm) wsum_partial4_kernel(int K, int T, int n_imp, int rows_per_cta,
                                                                  const float4 *__restrict__ eps,
                                                                  const float *__restrict__ w, float *part) {
  __shared__ float4 red4[2 * kWsThreads];  // (sums, corrections) of each thread
  __shared__ float2 wred[kWsThreads / 32];
  const int W4 = T / 2;                                  // float4 per row
  const int TC = W4 < kWsThreads ? W4 : kWsThreads;     // columns handled at once
  const int R = kWsThreads / TC;                         // row groups
  const int tid = threadIdx.x, c = tid % TC, ry = tid / TC;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(K, r0 + rows_per_cta);
  const int PS = ws_stride(T);
  float *rec = part + (size_t)blockIdx.x * PS;
  CSum wi;
  for (int k = r0 + tid; k < min(r1, n_imp); k += kWsThreads) wi.add(__ldg(w + k));
  wi = csum_warp(wi);
  if ((tid & 31) == 0) wred[tid >> 5] = make_float2(wi.s, wi.c);
  __syncthreads();
  if (tid == 0) {
    CSum sw;
    for (int g = 0; g < kWsThreads / 32; ++g) sw.add(CSum{wred[g].x, wred[g].y});
    rec[2 * T] = sw.value();
  }
  for (int cb = 0; cb < W4; cb += TC) {
    const int col = cb + c;
    CSum a[4];
    if (ry < R && col < W4) {
      const size_t stride = (size_t)R * W4;
      // blocks of kWsBlock rows: plain FMAs (loads in flight), then one compensated step per block
      for (int kb = r0 + ry; kb < r1; kb += kWsBlock * R) {
        const float4 *p = eps + (size_t)kb * W4 + col;
        float4 ev[kWsBlock];
        float wv[kWsBlock];
#pragma unroll
        for (int u = 0; u < kWsBlock; ++u) {  // every load of the block in flight
          const bool in = kb + u * R < r1;
          wv[u] = in ? __ldg(w + kb + u * R) : 0.0f;
          ev[u] = in ? __ldcs(p + u * stride) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // streamed once
        }
        float4 blk = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < kWsBlock; ++u) {
          blk.x = fmaf(wv[u], ev[u].x, blk.x);
          blk.y = fmaf(wv[u], ev[u].y, blk.y);
          blk.z = fmaf(wv[u], ev[u].z, blk.z);
          blk.w = fmaf(wv[u], ev[u].w, blk.w);
        }
        a[0].add(blk.x);
        a[1].add(blk.y);
        a[2].add(blk.z);
        a[3].add(blk.w);
      }
    }
    red4[2 * tid] = make_float4(a[0].s, a[1].s, a[2].s, a[3].s);
    red4[2 * tid + 1] = make_float4(a[0].c, a[1].c, a[2].c, a[3].c);
    __syncthreads();
    if (ry == 0 && col < W4) {
      CSum q[4];
      for (int g = 0; g < R; ++g) {
        const float4 os = red4[2 * (g * TC + c)], oc = red4[2 * (g * TC + c) + 1];
        q[0].add(CSum{os.x, oc.x});
        q[1].add(CSum{os.y, oc.y});
        q[2].add(CSum{os.z, oc.z});
        q[3].add(CSum{os.w, oc.w});
      }
      // records start on 16-byte boundaries
      reinterpret_cast<float4 *>(rec)[col] = make_float4(q[0].value(), q[1].value(), q[2].value(), q[3].value());
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
  __shared__ float2 red[kWfGroups][kWfCols + 1];
  __shared__ float2 redw[kWfGroups][kWfCols + 1];
  const int c = threadIdx.x % kWfCols, g = threadIdx.x / kWfCols;
  const int e = blockIdx.x * kWfCols + c;
  const int PS = ws_stride(T);
  CSum s, w_imp;
  if (e < 2 * T) {
#pragma unroll 8
    for (int b = g; b < n_cta; b += kWfGroups) {
      s.add(part[(size_t)b * PS + e]);
      w_imp.add(part[(size_t)b * PS + 2 * T]);
    }
  }
  red[g][c] = make_float2(s.s, s.c);
  redw[g][c] = make_float2(w_imp.s, w_imp.c);
  __syncthreads();
  if (g == 0 && e < 2 * T) {
    CSum st, wt;
    for (int q = 0; q < kWfGroups; ++q) {
      st.add(CSum{red[q][c].x, red[q][c].y});
      wt.add(CSum{redw[q][c].x, redw[q][c].y});
    }
    U_out[e] = fmaf(__ldg(U + e), wt.value(), st.value());
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
    wsum_partial_kernel<<<n_cta, kWsThreads, 2 * sizeof(float2) * kWsThreads, s>>>(
        K, T, n_imp, rows, reinterpret_cast<const float2 *>(eps), w, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wsum_final_kernel<<<(2 * T + kWfCols - 1) / kWfCols, kWsThreads, 0, s>>>(n_cta, T, part, U, U_out);
  return cudaGetLastError();
}

}  // namespace itmpc
