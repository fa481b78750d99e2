// itmpc_sum.cuh -- compensated FP32 summation for the normaliser and the
// weighted sums of Alg. 2 and the control law of Sec. III-D.
//
// The iteration forms eta~ = sum_k e_k, the importance-only sum, sum_k e_k^2,
// the running cost S_k = sum_t c_t and E = sum_k e_k eps_k in FP32.  Every such
// sum is carried as an unevaluated pair (s, c): s the running FP32 sum, c the
// accumulated rounding errors of the additions (Neumaier's variant of Kahan
// summation, Neumaier 1974), and products enter with their exact rounding error
// from one FMA (Ogita, Rump and Oishi 2005, "Accurate sum and dot product":
// TwoProduct).  Partial pairs are merged with Knuth's branch-free TwoSum, so a
// warp tree or a merge of records keeps the same error bound as one serial loop:
// about one rounding of the final value plus n u^2 |sum|, instead of n u |sum|.
//
// The compiler may not reassociate these operations (no fast-math flags), and
// products are formed with __fmul_rn so that they are not contracted into FMAs.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace itmpc {

// a + b = s + e exactly (Knuth, TAOCP vol. 2, 4.2.2: six operations, no branch).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

struct CSum {
  float s = 0.0f, c = 0.0f;

  // Neumaier step: the rounding error of s + x is recovered from whichever of
  // the two operands is larger in magnitude.
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float err = fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    c = __fadd_rn(c, err);
    s = t;
  }
  // a * b = p + q exactly (one FMA recovers q); both parts are accumulated.
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float q = fmaf(a, b, -p);
    add(p);
    c = __fadd_rn(c, q);
  }
  // merge another pair into this one
  __device__ __forceinline__ void add(const CSum &o) {
    float e;
    s = two_sum(s, o.s, e);
    c = __fadd_rn(__fadd_rn(c, o.c), e);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// Butterfly merge of the lanes' pairs; every lane ends with the warp's pair.
__device__ __forceinline__ CSum csum_warp(CSum v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    CSum w;
    w.s = __shfl_xor_sync(mask, v.s, o);
    w.c = __shfl_xor_sync(mask, v.c, o);
    v.add(w);
  }
  return v;
}

// The same over groups of `width` consecutive lanes (width a power of two <= 32).
__device__ __forceinline__ CSum csum_lanes(CSum v, int width) {
  for (int o = 1; o < width; o <<= 1) {
    CSum w;
    w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
    w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
    v.add(w);
  }
  return v;
}

// Compensated warp sum of one value per lane.
__device__ __forceinline__ float warp_csum(float x) {
  CSum v;
  v.s = x;
  return csum_warp(v).value();
}

}  // namespace itmpc
