// closed_loop.cu -- the end of Alg. 1's outer loop on the GPU: control smoothing
// (Sec. III-E, "Control Smoothing"), the first control to the actuators, and the
// warm start of the next iteration.
//
// For each item (one MPC instance) one CTA:
//   U_s = U'                       smoothing 0
//   U_s = SGF(U')                  smoothing 1 (the text: filter the weighted mean)
//   U_s = U + SGF(U' - U)          smoothing 2 (Alg. 1: U <- U + SGF * sum_k w_k eps_k)
// where SGF is the 5-point quadratic Savitzky-Golay filter (Savitzky & Golay 1964;
// convolution weights (-3, 12, 17, 12, -3)/35) with the end values replicated at the
// edges; u_applied = U_s[0]; when a plant state is given, x <- F(x, g(u_applied))
// with the context's network (noise-free Euler step of Sec. V-B); and
// U[t - 1] <- U_s[t], U[T - 1] <- (0, 0) (Initialize in the paper's parameter table).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "itmpc_device.cuh"
#include "itmpc_units.cuh"

namespace itmpc {

namespace {

constexpr int kLoopThreads = 128;

__device__ __forceinline__ float sgf5(const float *x, int n, int j) {
  auto at = [&](int i) { return x[2 * min(max(i, 0), n - 1)]; };
  return (-3.0f * at(j - 2) + 12.0f * at(j - 1) + 17.0f * at(j) + 12.0f * at(j + 1) - 3.0f * at(j + 2)) *
         (1.0f / 35.0f);
}

template <int ACT>
__global__ void __launch_bounds__(kLoopThreads) loop_kernel(const LoopItem *items, const LoopItem one, int H,
                                                            const float *__restrict__ net, const IterParams p,
                                                            int smoothing, int plant,
                                                            unsigned long long *counter,
                                                            const float *__restrict__ theta) {
  extern __shared__ __align__(16) float sm[];
  const LoopItem it = items ? items[blockIdx.x] : one;
  const int T = it.T, tid = threadIdx.x;
  float *Up = sm;            // U'  (T x 2)
  float *D = sm + 2 * T;     // U' - U, or U'
  float *Us = D + 2 * T;     // smoothed sequence
  float *hv = Us + 2 * T;    // hidden activations (H), then layer-2 outputs (H)
  float *h2 = hv + H;
  for (int i = tid; i < 2 * T; i += kLoopThreads) {
    const float up = it.U_prime[i];
    Up[i] = up;
    D[i] = smoothing == 2 ? up - it.U[i] : up;
  }
  __syncthreads();
  for (int i = tid; i < 2 * T; i += kLoopThreads) {
    const int t = i >> 1, c = i & 1;
    float v = smoothing == 0 ? Up[i] : sgf5(D + c, T, t);
    if (smoothing == 2) v += it.U[i];
    Us[i] = v;
  }
  __syncthreads();
  const float u0 = Us[0], u1 = Us[1];
  if (tid == 0 && it.u_applied) {
    it.u_applied[0] = u0;
    it.u_applied[1] = u1;
  }
  // warm start: slide the sequence down, Initialize(u_{T-1}) = (0, 0)
  for (int i = tid; i < 2 * T; i += kLoopThreads) it.U[i] = i + 2 < 2 * T ? Us[i + 2] : 0.0f;
  if (plant && it.x) {
    // x <- F(x, g(u_0)): network f(x_d, g) of Sec. V-B and Euler kinematics from the old state
    float x[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) x[q] = it.x[q];
    const float z[6] = {x[3], x[4], x[5], x[6], fminf(fmaxf(u0, p.umin0), p.umax0),
                        fminf(fmaxf(u1, p.umin1), p.umax1)};
    if (theta) {  // the basis-function model
      if (tid == 0) {
        BasisDyn B;
        for (int i = 0; i < 100; ++i) B.theta[i] = theta[i];
        float d[4];
        B.eval(z[0], z[1], z[2], z[3], z[4], z[5], d[0], d[1], d[2], d[3]);
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        it.x[0] = x[0] + (cs * x[4] - sn * x[5]) * p.dt;
        it.x[1] = x[1] + (sn * x[4] + cs * x[5]) * p.dt;
        it.x[2] = x[2] + x[6] * p.dt;
#pragma unroll
        for (int q = 0; q < 4; ++q) it.x[3 + q] = x[3 + q] + d[q] * p.dt;
      }
    } else {
    for (int j = tid; j < H; j += kLoopThreads) {
      float a = __ldg(net + net_off_b1(H) + j);
#pragma unroll
      for (int m = 0; m < 6; ++m) a = fmaf(__ldg(net + net_off_W1(H) + j * 6 + m), z[m], a);
      hv[j] = activation<ACT>(a);
    }
    __syncthreads();
    for (int j = tid; j < H; j += kLoopThreads) {
      // four independent chains so that the row's weight loads are in flight together
      const float *wr = net + net_off_W2(H) + (size_t)j * H;
      float a0 = __ldg(net + net_off_b2(H) + j), a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 8
      for (int i = 0; i < H; i += 4) {
        a0 = fmaf(__ldg(wr + i), hv[i], a0);
        a1 = fmaf(__ldg(wr + i + 1), hv[i + 1], a1);
        a2 = fmaf(__ldg(wr + i + 2), hv[i + 2], a2);
        a3 = fmaf(__ldg(wr + i + 3), hv[i + 3], a3);
      }
      h2[j] = activation<ACT>((a0 + a1) + (a2 + a3));
    }
    __syncthreads();
    if (tid < 32) {
      float d[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float a = 0.0f;
        for (int j = tid; j < H; j += 32) a = fmaf(__ldg(net + net_off_W3(H) + o * H + j), h2[j], a);
        d[o] = warp_sum(a) + __ldg(net + net_off_b3(H) + o);
      }
      if (tid == 0) {
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        it.x[0] = x[0] + (cs * x[4] - sn * x[5]) * p.dt;
        it.x[1] = x[1] + (sn * x[4] + cs * x[5]) * p.dt;
        it.x[2] = x[2] + x[6] * p.dt;
#pragma unroll
        for (int q = 0; q < 4; ++q) it.x[3 + q] = x[3 + q] + d[q] * p.dt;
      }
    }
    }
  }
  // the next replay of a captured loop draws the next iteration's noise
  if (counter && blockIdx.x == 0 && tid == 0) *counter += 1ull;
}

}  // namespace

cudaError_t loop_launch(const LoopItem *items_dev, const LoopItem *item_host, int n, int H, const float *net,
                        const IterParams &p, int smoothing, int plant, unsigned long long *counter, cudaStream_t s,
                        const float *theta) {
  if (n <= 0) return cudaSuccess;
  int T_max = 0;
  if (items_dev) T_max = p.T;  // callers pass the largest horizon in p.T for a batch
  else T_max = item_host->T;
  const size_t smem = sizeof(float) * (6 * (size_t)T_max + 2 * (size_t)H);
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = p.activation == 1
            ? cudaFuncSetAttribute(loop_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(loop_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const LoopItem one = item_host ? *item_host : LoopItem{};
  if (p.activation == 1)
    loop_kernel<1><<<n, kLoopThreads, smem, s>>>(items_dev, one, H, net, p, smoothing, plant, counter, theta);
  else
    loop_kernel<0><<<n, kLoopThreads, smem, s>>>(items_dev, one, H, net, p, smoothing, plant, counter, theta);
  return cudaGetLastError();
}

}  // namespace itmpc
