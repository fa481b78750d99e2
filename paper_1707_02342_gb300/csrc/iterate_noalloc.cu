// iterate_noalloc.cu -- itmpc_iterate_noalloc: one FP32 control iteration that
// allocates no device memory.
//
// Some callers cannot allocate GPU memory at the time they run an iteration:
// a real-time control loop that forbids allocation after start-up (cudaMalloc
// may synchronise the whole device and has no latency bound), or a plug-in
// inside an application that has already reserved all device memory for its
// own pool.  This entry point serves them.  The caller passes every input and
// output as a device pointer; the scratch the fused kernel needs (packed
// network, per-CTA partial records, merge counters, costs when the caller
// passes none, diagnostics) lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "itmpc.h"
#include "itmpc_internal.h"

using namespace itmpc;

namespace {

// 4 MiB of scratch, shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ITMPC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device
size_t g_smem_optin[kMaxDevices] = {};

// First call on a device (with that device current): resolve the array's
// device address.  Host code may not use the symbol itself as a pointer.
itmpc_status setup_device(int dev, void **ptr, size_t *smem) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ITMPC_ERR_CUDA;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return ITMPC_ERR_CUDA;
    }
    g_smem_optin[dev] = (size_t)optin;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  *smem = g_smem_optin[dev];
  return ITMPC_OK;
}

bool fin(float v) { return isfinite(v) != 0; }

itmpc_status check(const itmpc_config *c) {
  if (!c) return ITMPC_ERR_ARG;
  if (c->K < 1 || c->K > ITMPC_NOALLOC_MAX_K || c->T < 1 || c->T > ITMPC_NOALLOC_MAX_T) return ITMPC_ERR_ARG;
  if (c->hidden != 32 && c->hidden != 64 && c->hidden != 128) return ITMPC_ERR_ARG;
  if (!(c->lambda > 0.f) || !fin(c->lambda) || !fin(c->dt) || !fin(c->gamma)) return ITMPC_ERR_ARG;
  if (!(c->alpha_explore >= 0.f && c->alpha_explore <= 1.f)) return ITMPC_ERR_ARG;
  for (int i = 0; i < 2; ++i)
    if (!(c->sigma[i] >= 0.f) || !fin(c->sigma[i]) || !(c->u_min[i] <= c->u_max[i])) return ITMPC_ERR_ARG;
  if (c->gamma != 0.f && (c->sigma[0] == 0.f || c->sigma[1] == 0.f)) return ITMPC_ERR_ARG;
  for (int i = 0; i < 4; ++i)
    if (!fin(c->cost_w[i])) return ITMPC_ERR_ARG;
  if (!(c->crash_decay > 0.f) || !fin(c->crash_decay)) return ITMPC_ERR_ARG;
  if (c->precision != ITMPC_FP32) return ITMPC_ERR_ARG;
  if (c->dynamics != ITMPC_DYN_NETWORK) return ITMPC_ERR_ARG;  // the fused kernel runs the network
  if (c->activation != ITMPC_ACT_TANH && c->activation != ITMPC_ACT_IDENTITY) return ITMPC_ERR_ARG;
  return ITMPC_OK;
}

size_t round_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

}  // namespace

extern "C" itmpc_status itmpc_iterate_noalloc(const itmpc_config *cfg, const float *const *W, const float *const *b,
                                              const float *map, int32_t width, int32_t height, float res,
                                              float origin_x, float origin_y, const float *x0, const float *U,
                                              uint64_t iter, float *U_out, float *weights, float *costs) {
  itmpc_status st = check(cfg);
  if (st != ITMPC_OK) return st;
  if (!W || !b || !map || !x0 || !U || !U_out || width < 1 || height < 1 || !(res > 0.f) || !fin(res) ||
      !fin(origin_x) || !fin(origin_y))
    return ITMPC_ERR_ARG;
  for (int l = 0; l < 3; ++l)
    if (!W[l] || !b[l]) return ITMPC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ITMPC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return ITMPC_ERR_CUDA;
  void *base = nullptr;
  size_t smem_limit = 0;
  st = setup_device(dev, &base, &smem_limit);
  if (st != ITMPC_OK) return st;

  const int K = cfg->K, T = cfg->T, H = cfg->hidden;
  const Fp32Tile tile = fp32_pick_tile(K, T, H, smem_limit);
  if (fp32_smem_bytes(T, H, tile) > smem_limit) return ITMPC_ERR_ARG;
  const int nC = fp32_num_ctas(K, tile);
  const int nG = (nC + tile.group - 1) / tile.group;
  const size_t PL = (size_t)partial_len(T);

  // carve the scratch: every region 256-byte aligned
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = round_up(off + bytes, 256);
    return (unsigned char *)base + at;
  };
  float *net = (float *)take(sizeof(float) * (size_t)net_floats(H));
  float *cost_buf = (float *)take(sizeof(float) * (size_t)K);
  float *partials = (float *)take(sizeof(float) * PL * (size_t)nC);
  float *group_rec = (float *)take(sizeof(float) * PL * (size_t)nG);
  float *stats = (float *)take(sizeof(float) * ITMPC_STATS_LEN);
  unsigned int *counters = (unsigned int *)take(sizeof(unsigned int) * (size_t)(1 + nG + 2));
  int *status = (int *)take(sizeof(int));
  // With GB300's 227 KB of shared memory per block the tile picker's CTAs keep
  // every size within the stated limits under about 2.2 MB of scratch.  A GPU
  // with less shared memory per block gets smaller CTAs, hence more records, and
  // the largest sizes can exceed the array: they are refused here.
  if (off > (size_t)ITMPC_NOALLOC_SCRATCH_BYTES) return ITMPC_ERR_ARG;

  cudaStream_t s = (cudaStream_t)cfg->stream;
  const size_t nW[3] = {(size_t)6 * H, (size_t)H * H, (size_t)4 * H};
  const size_t nb[3] = {(size_t)H, (size_t)H, 4};
  const size_t offW[3] = {(size_t)net_off_W1(H), (size_t)net_off_W2(H), (size_t)net_off_W3(H)};
  const size_t offb[3] = {(size_t)net_off_b1(H), (size_t)net_off_b2(H), (size_t)net_off_b3(H)};
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = cudaMemcpyAsync(net + offW[l], W[l], sizeof(float) * nW[l], cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net + offb[l], b[l], sizeof(float) * nb[l], cudaMemcpyDeviceToDevice, s);
  }
  // the scratch keeps the previous call's contents: the counters and the status must start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(unsigned int) * (size_t)(1 + nG + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ITMPC_ERR_CUDA;
  }

  IterParams p{};
  p.K = K;
  p.T = T;
  p.H = H;
  p.activation = cfg->activation;
  const double nimp = ceil((1.0 - (double)cfg->alpha_explore) * (double)K);
  p.n_imp = (int)(nimp < 0 ? 0 : (nimp > K ? K : nimp));
  p.ctr2 = (uint32_t)iter;
  p.ctr3 = (uint32_t)((iter >> 32) & 0xFFFFu) | (cfg->instance << 16);
  p.key0 = (uint32_t)cfg->seed;
  p.key1 = (uint32_t)(cfg->seed >> 32);
  p.sigma0 = cfg->sigma[0];
  p.sigma1 = cfg->sigma[1];
  p.dt = cfg->dt;
  p.umin0 = cfg->u_min[0]; p.umin1 = cfg->u_min[1];
  p.umax0 = cfg->u_max[0]; p.umax1 = cfg->u_max[1];
  p.w_track = cfg->cost_w[0]; p.w_speed = cfg->cost_w[1]; p.w_stab = cfg->cost_w[2]; p.w_crash = cfg->cost_w[3];
  p.v_des = cfg->v_des;
  p.crash_cost = cfg->crash_cost;
  p.log2_decay = (float)log2((double)cfg->crash_decay);
  p.track_thresh = cfg->track_thresh;
  p.slip_thresh = cfg->slip_thresh;
  p.map_cap = cfg->map_cap;
  p.gamma = cfg->gamma;
  p.inv_sig2_0 = cfg->sigma[0] > 0 ? (float)(1.0 / ((double)cfg->sigma[0] * cfg->sigma[0])) : 0.f;
  p.inv_sig2_1 = cfg->sigma[1] > 0 ? (float)(1.0 / ((double)cfg->sigma[1] * cfg->sigma[1])) : 0.f;
  p.lambda = cfg->lambda;
  p.inv_lambda = (float)(1.0 / (double)cfg->lambda);
  p.map = map;
  p.map_w = width;
  p.map_h = height;
  p.inv_res = (float)(1.0 / (double)res);
  p.origin_x = origin_x;
  p.origin_y = origin_y;
  p.net = net;
  p.x0 = x0;
  p.U = U;
  p.U_out = U_out;
  p.weights = weights;
  p.weights_inline = 1;  // K <= ITMPC_NOALLOC_MAX_K: the merging CTA writes the weights
  p.costs = costs ? costs : cost_buf;
  p.partials = partials;
  p.group_rec = group_rec;
  p.counters = counters;
  p.grid_bar = counters + 1 + nG;
  p.stats = stats;
  p.status = status;
  e = fp32_launch_iterate(p, tile, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ITMPC_ERR_CUDA;
  }
  int dev_status = 0;
  e = cudaMemcpyAsync(&dev_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ITMPC_ERR_CUDA;
  }
  return dev_status == 0 ? ITMPC_OK : (itmpc_status)dev_status;
}
