// itmpc_api.cu -- the C ABI of include/itmpc.h: argument checks, context-owned
// device memory, launches.  All arithmetic of the iteration is in the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "itmpc.h"
#include "itmpc_internal.h"

using namespace itmpc;

struct itmpc_ctx {
  itmpc_config cfg{};
  int K_cap = 0, T_max = 0, H = 0, device = -1;
  cudaStream_t stream = nullptr;
  float *net = nullptr;
  bool have_net = false;
  std::vector<float> net_host;  // host copy of the packed network (kernel-parameter weights)
  float *map = nullptr;         // n_maps maps of map_w x map_h, contiguous
  int map_w = 0, map_h = 0, n_maps = 0;
  float res = 1.f, origin_x = 0.f, origin_y = 0.f;
  bool have_map = false;
  float *partials = nullptr, *group_rec = nullptr, *scale = nullptr, *costs = nullptr, *stats = nullptr;
  unsigned int *counters = nullptr;
  size_t n_counters = 0;
  int *status = nullptr;
  // device staging for the host-pointer entry point
  float *x0_d = nullptr, *U_d = nullptr, *Uout_d = nullptr, *w_d = nullptr;
  size_t smem_optin = 0;
  // batched iterations (itmpc_reserve_batch)
  int batch_max_inst = 0, batch_max_units = 0;
  int64_t batch_max_samples = 0;
  TpsInstance *inst_d = nullptr, *inst_h = nullptr;
  TpsUnit *units_d = nullptr, *units_h = nullptr;
  float *batch_partials = nullptr, *batch_costs = nullptr, *batch_stats = nullptr;
  unsigned int *unit_counter = nullptr;
  cudaEvent_t staged = nullptr;  // the last H2D copy of the staging buffers
  // tensor-core operand images of the H = 128 network: [0] BF16, [1] FP8 layer 2
  unsigned char *tc_img[2] = {nullptr, nullptr};
  // adjoint form (itmpc_reserve_adjoint): per-CTA gradient records and 4 scalars
  float *adj_part = nullptr, *adj_scal = nullptr;
  float *cem_scal = nullptr;  // cross-entropy threshold and elite count of the last CEM iteration
  float *wsum_part = nullptr;  // records of the update from materialised noise
  int sms = 0;
  // host-pointer iterations as one captured graph: upload of (x0, iter, U), the fused
  // iteration, download of (U', status); pinned host and device blocks of the same layout
  cudaGraphExec_t host_exec = nullptr;
  unsigned char *hblk_in = nullptr, *dblk_in = nullptr, *hblk_out = nullptr, *dblk_out = nullptr;
  bool host_mapped = false;  // the host graph's kernel writes U' and the status into hblk_out itself
  // basis-function dynamics model: coefficients (host copy for the kernel parameters, device copy)
  std::vector<float> theta_host;
  float *theta_d = nullptr;
  bool have_theta = false;
  // batched form: FP32 launch shape (itmpc_autotune_batch) and the captured closed-loop graph
  TpsTile tps_tile{kTpsThreads, 0};
  cudaGraphExec_t graph_exec = nullptr;
  TpsInstance *ginst_d = nullptr;
  TpsUnit *gunits_d = nullptr;
  LoopItem *gloop_d = nullptr;  // the batched graph's closed-loop items
  // single-instance closed-loop graph (itmpc_control_graph_create) and its iteration counter
  cudaGraphExec_t loop_exec = nullptr;
  unsigned long long *loop_ctr = nullptr;
  std::string err;
};

namespace {

const char *kNoCtx = "no context";

itmpc_status fail(itmpc_ctx *c, itmpc_status st, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

itmpc_status cuda_fail(itmpc_ctx *c, cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a sticky-free error so later calls are not affected
  return fail(c, e == cudaErrorMemoryAllocation ? ITMPC_ERR_OOM : ITMPC_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(c, call, what)                         \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

bool finite(float v) { return isfinite(v) != 0; }

// Host-side validation of a configuration (no CUDA calls).
itmpc_status check_config(const itmpc_config *cfg, char *msg, size_t n) {
  if (!cfg) { snprintf(msg, n, "cfg is NULL"); return ITMPC_ERR_ARG; }
  const int T_max = cfg->T_max > 0 ? cfg->T_max : cfg->T;
  if (cfg->K < 1 || cfg->K > ITMPC_MAX_K) { snprintf(msg, n, "K=%d outside [1, %d]", cfg->K, ITMPC_MAX_K); return ITMPC_ERR_ARG; }
  if (cfg->T < 1 || T_max > ITMPC_MAX_T || cfg->T > T_max) {
    snprintf(msg, n, "T=%d / T_max=%d outside 1 <= T <= T_max <= %d", cfg->T, cfg->T_max, ITMPC_MAX_T);
    return ITMPC_ERR_ARG;
  }
  if (cfg->hidden != 32 && cfg->hidden != 64 && cfg->hidden != 128) {
    snprintf(msg, n, "hidden=%d not one of 32, 64, 128", cfg->hidden);
    return ITMPC_ERR_ARG;
  }
  if (!(cfg->lambda > 0.f) || !finite(cfg->lambda)) { snprintf(msg, n, "lambda must be finite and > 0"); return ITMPC_ERR_ARG; }
  if (!finite(cfg->dt) || !finite(cfg->gamma)) { snprintf(msg, n, "dt and gamma must be finite"); return ITMPC_ERR_ARG; }
  if (!(cfg->alpha_explore >= 0.f && cfg->alpha_explore <= 1.f)) { snprintf(msg, n, "alpha_explore outside [0, 1]"); return ITMPC_ERR_ARG; }
  for (int i = 0; i < 2; ++i) {
    if (!(cfg->sigma[i] >= 0.f) || !finite(cfg->sigma[i])) { snprintf(msg, n, "sigma[%d] must be finite and >= 0", i); return ITMPC_ERR_ARG; }
    if (!(cfg->u_min[i] <= cfg->u_max[i])) { snprintf(msg, n, "u_min[%d] > u_max[%d]", i, i); return ITMPC_ERR_ARG; }
  }
  if (cfg->gamma != 0.f && (cfg->sigma[0] == 0.f || cfg->sigma[1] == 0.f)) {
    snprintf(msg, n, "gamma != 0 needs sigma > 0 (Sigma^-1 in the control cost)");
    return ITMPC_ERR_ARG;
  }
  for (int i = 0; i < 4; ++i)
    if (!finite(cfg->cost_w[i])) { snprintf(msg, n, "cost_w[%d] not finite", i); return ITMPC_ERR_ARG; }
  if (!(cfg->crash_decay > 0.f) || !finite(cfg->crash_decay)) { snprintf(msg, n, "crash_decay must be > 0"); return ITMPC_ERR_ARG; }
  if (cfg->precision != ITMPC_FP32 && cfg->precision != ITMPC_BF16 && cfg->precision != ITMPC_FP8) {
    snprintf(msg, n, "unknown precision %d", cfg->precision);
    return ITMPC_ERR_ARG;
  }
  if (cfg->dynamics != ITMPC_DYN_NETWORK && cfg->dynamics != ITMPC_DYN_BASIS) {
    snprintf(msg, n, "unknown dynamics model %d", cfg->dynamics);
    return ITMPC_ERR_ARG;
  }
  if (cfg->dynamics == ITMPC_DYN_BASIS && cfg->precision != ITMPC_FP32) {
    snprintf(msg, n, "the basis-function model runs in FP32 only");
    return ITMPC_ERR_ARG;
  }
  if (cfg->precision != ITMPC_FP32 && cfg->hidden != kTcHidden) {
    snprintf(msg, n, "BF16 / FP8 iterations need hidden == %d", kTcHidden);
    return ITMPC_ERR_ARG;
  }
  if (cfg->activation != ITMPC_ACT_TANH && cfg->activation != ITMPC_ACT_IDENTITY) { snprintf(msg, n, "bad activation"); return ITMPC_ERR_ARG; }
  return ITMPC_OK;
}

IterParams make_params(const itmpc_ctx *c) {
  const itmpc_config &g = c->cfg;
  IterParams p{};
  p.K = g.K;
  p.T = g.T;
  p.H = c->H;
  p.activation = g.activation;
  // Alg. 1: sample k is centred on U iff k < (1 - alpha) K, i.e. k < ceil((1 - alpha) K)
  double nimp = ceil((1.0 - (double)g.alpha_explore) * (double)g.K);
  p.n_imp = (int)(nimp < 0 ? 0 : (nimp > g.K ? g.K : nimp));
  p.key0 = (uint32_t)g.seed;
  p.key1 = (uint32_t)(g.seed >> 32);
  p.sigma0 = g.sigma[0];
  p.sigma1 = g.sigma[1];
  p.dt = g.dt;
  p.umin0 = g.u_min[0]; p.umin1 = g.u_min[1];
  p.umax0 = g.u_max[0]; p.umax1 = g.u_max[1];
  p.w_track = g.cost_w[0]; p.w_speed = g.cost_w[1]; p.w_stab = g.cost_w[2]; p.w_crash = g.cost_w[3];
  p.v_des = g.v_des;
  p.crash_cost = g.crash_cost;
  p.log2_decay = (float)log2((double)g.crash_decay);
  p.track_thresh = g.track_thresh;
  p.slip_thresh = g.slip_thresh;
  p.map_cap = g.map_cap;
  p.gamma = g.gamma;
  p.inv_sig2_0 = g.sigma[0] > 0 ? (float)(1.0 / ((double)g.sigma[0] * g.sigma[0])) : 0.f;
  p.inv_sig2_1 = g.sigma[1] > 0 ? (float)(1.0 / ((double)g.sigma[1] * g.sigma[1])) : 0.f;
  p.lambda = g.lambda;
  p.inv_lambda = (float)(1.0 / (double)g.lambda);
  p.map = c->map;
  p.map_w = c->map_w;
  p.map_h = c->map_h;
  p.inv_res = (float)(1.0 / (double)c->res);
  p.origin_x = c->origin_x;
  p.origin_y = c->origin_y;
  p.net = c->net;
  p.costs = c->costs;
  p.partials = c->partials;
  p.group_rec = c->group_rec;
  p.counters = c->counters;
  p.grid_bar = c->counters + (c->n_counters - 2);
  p.stats = c->stats;
  p.status = c->status;
  p.states_every = 1;
  return p;
}

void set_iter(IterParams &p, uint64_t iter, uint32_t instance) {
  p.ctr2 = (uint32_t)iter;
  p.ctr3 = (uint32_t)((iter >> 32) & 0xFFFFu) | (instance << 16);
}

itmpc_status ready(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  if (c->cfg.dynamics == ITMPC_DYN_BASIS) {
    if (!c->have_theta) return fail(c, ITMPC_ERR_STATE, "itmpc_set_basis has not been called");
  } else if (!c->have_net) {
    return fail(c, ITMPC_ERR_STATE, "itmpc_set_dynamics has not been called");
  }
  if (!c->have_map) return fail(c, ITMPC_ERR_STATE, "itmpc_set_costmap has not been called");
  return ITMPC_OK;
}

// Host-graph blocks: in = [x0 (8 floats), iteration index (uint64), pad, U (2 T_max)], copied
// to the device by the graph; out = [U' (2 T_max), status (int), pad], written by the kernel
// straight into the pinned block (mapped into the device's address space), or copied back
// where the block cannot be mapped.
constexpr size_t kHinU = 48;  // byte offset of U in the input block (16-byte aligned)
size_t hin_bytes(int T_max) { return kHinU + sizeof(float) * 2 * (size_t)T_max; }
size_t hout_status(int T_max) { return sizeof(float) * 2 * (size_t)T_max; }
size_t hout_bytes(int T_max) { return (hout_status(T_max) + sizeof(int) + 15) & ~size_t(15); }

void drop_host_graph(itmpc_ctx *c) {
  if (c->host_exec) {
    cudaGraphExecDestroy(c->host_exec);
    c->host_exec = nullptr;
  }
}

constexpr int kTpsMinK = 4096;   // from here on one thread per sample beats a warp per sample (H = 32)
constexpr int kWideMinK = 2048;  // from here on the tiled GEMM kernel beats a warp per sample (H = 64, 128)

// Batched contexts: the thread-per-sample FP32 kernels (H = 32), the tiled FP32 kernels
// (H = 64, 128) and the tensor-core kernels (H = 128).
bool batch_capable(int H) { return H == 32 || H == 64 || H == kTcHidden; }

// Smallest work unit any kernel of this width may use: batch buffers are sized for it.
int min_unit(int H) { return H == 32 ? kTpsMinUnit : wide_unit_samples(H); }

// Single iterations that run as a batch of one instance.
bool single_as_batch(const itmpc_ctx *c, bool debug_out);

}  // namespace

extern "C" itmpc_status itmpc_reserve_batch(itmpc_ctx *c, int32_t max_instances, int64_t max_total_samples);

namespace {

// One shard of a sample-sharded iteration: the context's samples are global samples
// k_base .. k_base + K - 1, the exploration split counts n_imp global samples, and the merged
// partial record goes to rec_out instead of U', the weights and the stats.
struct ShardSpec {
  uint32_t k_base;
  int n_imp;
  float *rec_out;
};

itmpc_status run_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, float *states, int n_states,
                       int states_every = 1, const ShardSpec *shard = nullptr);
itmpc_status run_batch_tile(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, float *states, int n_states,
                            TpsTile tile, int states_every = 1, const ShardSpec *shard = nullptr);
itmpc_status build_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, int nt, TpsInstance *inst_h,
                         TpsUnit *units_h, int *n_units);
TpsShared batch_shared(const itmpc_ctx *c, const TpsInstance *inst_d, const TpsUnit *units_d, int n, int n_units);
itmpc_status launch_batch(itmpc_ctx *c, const TpsShared &sh, TpsTile tile, cudaStream_t s);
itmpc_status batch_ready(itmpc_ctx *c);
int batch_nt(const itmpc_ctx *c);

itmpc_status run_iteration(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, float *U_out,
                           float *weights, float *costs, float *states, int n_states, float *eps_out,
                           int states_every = 1, const ShardSpec *shard = nullptr) {
  const bool tc = c->cfg.precision != ITMPC_FP32;
  if (tc || (!eps_out && single_as_batch(c, states != nullptr))) {
    // the tensor-core kernels, or many samples: the thread-per-sample kernels, as a batch of one instance
    if (eps_out) return fail(c, ITMPC_ERR_ARG, "noise output is not available for this precision");
    itmpc_instance q{};
    q.K = c->cfg.K;
    q.T = c->cfg.T;
    q.map_index = 0;
    q.instance = c->cfg.instance;
    q.iter = iter;
    q.x0 = x0;
    q.U = U;
    q.U_out = U_out;
    q.weights = weights;
    q.costs = costs ? costs : c->costs;
    q.stats = c->stats;
    return run_batch(c, 1, &q, states, n_states, states_every, shard);
  }
  IterParams p = make_params(c);
  set_iter(p, iter, c->cfg.instance);
  p.x0 = x0;
  p.U = U;
  p.U_out = U_out;
  p.weights = weights;
  p.weights_inline = c->cfg.K <= 16384;
  p.states_out = states;
  p.n_states = n_states;
  p.states_every = states_every;
  p.eps_out = eps_out;
  if (costs) p.costs = costs;  // write S_k straight into the caller's buffer
  if (shard) {
    p.k_base = shard->k_base;
    p.n_imp = shard->n_imp;
    p.rec_out = shard->rec_out;
    p.weights = nullptr;
  }
  const Fp32Tile tile = fp32_pick_tile(p.K, p.T, p.H, c->smem_optin);
  CK(c, fp32_launch_iterate(p, tile, c->stream), "fused FP32 iteration launch");
  if (weights && !p.weights_inline) CK(c, launch_finalize_weights(p, c->stream), "weights launch");
  return ITMPC_OK;
}

void free_ctx(itmpc_ctx *c) {
  float *bufs[] = {c->net,   c->map,   c->partials, c->group_rec, c->scale, c->costs,
                   c->stats, c->x0_d, c->U_d,      c->Uout_d,    c->w_d};
  for (float *b : bufs)
    if (b) cudaFree(b);
  if (c->counters) cudaFree(c->counters);
  if (c->status) cudaFree(c->status);
  void *bbufs[] = {c->inst_d, c->units_d, c->batch_partials, c->batch_costs, c->batch_stats, c->unit_counter};
  for (void *b : bbufs)
    if (b) cudaFree(b);
  if (c->inst_h) cudaFreeHost(c->inst_h);
  if (c->units_h) cudaFreeHost(c->units_h);
  if (c->staged) cudaEventDestroy(c->staged);
  for (unsigned char *b : c->tc_img)
    if (b) cudaFree(b);
  if (c->adj_part) cudaFree(c->adj_part);
  if (c->adj_scal) cudaFree(c->adj_scal);
  if (c->cem_scal) cudaFree(c->cem_scal);
  if (c->wsum_part) cudaFree(c->wsum_part);
  if (c->theta_d) cudaFree(c->theta_d);
  if (c->host_exec) cudaGraphExecDestroy(c->host_exec);
  if (c->dblk_in) cudaFree(c->dblk_in);
  if (c->dblk_out) cudaFree(c->dblk_out);
  if (c->hblk_in) cudaFreeHost(c->hblk_in);
  if (c->hblk_out) cudaFreeHost(c->hblk_out);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->ginst_d) cudaFree(c->ginst_d);
  if (c->gunits_d) cudaFree(c->gunits_d);
  if (c->gloop_d) cudaFree(c->gloop_d);
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->loop_ctr) cudaFree(c->loop_ctr);
  delete c;
}

}  // namespace

extern "C" {

itmpc_status itmpc_create(const itmpc_config *cfg, itmpc_ctx **out) {
  if (!out) return ITMPC_ERR_ARG;
  *out = nullptr;
  char msg[256];
  itmpc_status st = check_config(cfg, msg, sizeof msg);
  if (st != ITMPC_OK) return st;
  itmpc_ctx *c = new itmpc_ctx();
  c->cfg = *cfg;
  c->K_cap = cfg->K;
  c->T_max = cfg->T_max > 0 ? cfg->T_max : cfg->T;
  c->cfg.T_max = c->T_max;
  c->H = cfg->hidden;
  c->stream = (cudaStream_t)cfg->stream;
  auto bail = [&](cudaError_t e, const char *what) {
    cudaGetLastError();
    free_ctx(c);
    return e == cudaErrorMemoryAllocation ? ITMPC_ERR_OOM : ITMPC_ERR_CUDA;
    (void)what;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) return bail(e, "attribute");
  c->smem_optin = (size_t)optin;
  const Fp32Tile tile = fp32_pick_tile(c->K_cap, c->T_max, c->H, c->smem_optin);
  if (fp32_smem_bytes(c->T_max, c->H, tile) > c->smem_optin) {
    free_ctx(c);
    return ITMPC_ERR_ARG;
  }
  const Fp32Scratch sc = fp32_scratch(c->K_cap, c->T_max, c->H);
  struct { float **p; size_t n; } allocs[] = {
      {&c->net, (size_t)net_floats(c->H)}, {&c->partials, sc.partial_floats}, {&c->group_rec, sc.group_floats},
      {&c->scale, sc.scale_floats > 0 ? sc.scale_floats : 1}, {&c->costs, (size_t)c->K_cap},     {&c->stats, ITMPC_STATS_LEN},
      {&c->x0_d, 8},                       {&c->U_d, 2 * (size_t)c->T_max},   {&c->Uout_d, 2 * (size_t)c->T_max},
      {&c->w_d, (size_t)c->K_cap}};
  for (auto &a : allocs) {
    e = cudaMalloc((void **)a.p, sizeof(float) * a.n);
    if (e != cudaSuccess) return bail(e, "cudaMalloc");
  }
  c->n_counters = sc.counters;
  e = cudaMalloc((void **)&c->counters, sizeof(unsigned int) * c->n_counters);
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  e = cudaMalloc((void **)&c->status, sizeof(int));
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  e = cudaMalloc((void **)&c->cem_scal, sizeof(float) * 4);
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->wsum_part, sizeof(float) * wsum_part_floats(c->T_max, c->sms));
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  e = cudaMalloc((void **)&c->dblk_in, hin_bytes(c->T_max));
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->dblk_out, hout_bytes(c->T_max));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&c->hblk_in, hin_bytes(c->T_max));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&c->hblk_out, hout_bytes(c->T_max));
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  if (c->H == kTcHidden) {
    for (int i = 0; i < 2; ++i) {
      e = cudaMalloc((void **)&c->tc_img[i], tc_image_bytes(i + 1));
      if (e != cudaSuccess) return bail(e, "cudaMalloc");
    }
  }
  if ((c->H == 32 && c->K_cap >= kTpsMinK) || (c->H == 64 && c->K_cap >= kWideMinK) || c->H == kTcHidden ||
      cfg->dynamics == ITMPC_DYN_BASIS) {
    itmpc_status bs = itmpc_reserve_batch(c, 1, c->K_cap);
    if (bs != ITMPC_OK) {
      free_ctx(c);
      return bs;
    }
  }
  e = cudaMemset(c->counters, 0, sizeof(unsigned int) * c->n_counters);
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->stats, 0, sizeof(float) * ITMPC_STATS_LEN);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return bail(e, "init");
  *out = c;
  return ITMPC_OK;
}

itmpc_status itmpc_set_config(itmpc_ctx *c, const itmpc_config *cfg) {
  if (!c) return ITMPC_ERR_ARG;
  drop_host_graph(c);
  char msg[256];
  itmpc_status st = check_config(cfg, msg, sizeof msg);
  if (st != ITMPC_OK) return fail(c, st, "%s", msg);
  if (cfg->K > c->K_cap) return fail(c, ITMPC_ERR_ARG, "K=%d exceeds the K=%d the context was created for", cfg->K, c->K_cap);
  if (cfg->T > c->T_max) return fail(c, ITMPC_ERR_ARG, "T=%d exceeds T_max=%d", cfg->T, c->T_max);
  if (cfg->hidden != c->H) return fail(c, ITMPC_ERR_ARG, "hidden width cannot change (%d -> %d)", c->H, cfg->hidden);
  if (cfg->dynamics != c->cfg.dynamics) return fail(c, ITMPC_ERR_ARG, "the dynamics model cannot change");
  const int T_max = c->T_max;
  c->cfg = *cfg;
  c->cfg.T_max = T_max;
  c->stream = (cudaStream_t)cfg->stream;
  return ITMPC_OK;
}

itmpc_status itmpc_set_stream(itmpc_ctx *c, void *stream) {
  if (!c) return ITMPC_ERR_ARG;
  drop_host_graph(c);
  c->stream = (cudaStream_t)stream;
  c->cfg.stream = stream;
  return ITMPC_OK;
}

itmpc_status itmpc_set_dynamics(itmpc_ctx *c, int32_t n_layers, const int32_t *widths, const float *const *W,
                                const float *const *b, int32_t on_device) {
  if (!c) return ITMPC_ERR_ARG;
  if (n_layers != 3 || !widths || !W || !b) return fail(c, ITMPC_ERR_ARG, "need n_layers == 3 and non-NULL arrays");
  const int H = c->H;
  if (widths[0] != 6 || widths[1] != H || widths[2] != H || widths[3] != 4)
    return fail(c, ITMPC_ERR_ARG, "widths must be {6, %d, %d, 4}", H, H);
  for (int l = 0; l < 3; ++l)
    if (!W[l] || !b[l]) return fail(c, ITMPC_ERR_ARG, "layer %d pointer is NULL", l);
  const size_t nW[3] = {(size_t)6 * H, (size_t)H * H, (size_t)4 * H};
  const size_t nb[3] = {(size_t)H, (size_t)H, 4};
  const size_t offW[3] = {(size_t)net_off_W1(H), (size_t)net_off_W2(H), (size_t)net_off_W3(H)};
  const size_t offb[3] = {(size_t)net_off_b1(H), (size_t)net_off_b2(H), (size_t)net_off_b3(H)};
  for (int l = 0; l < 3; ++l) {
    if (on_device) {
      CK(c, cudaMemcpyAsync(c->net + offW[l], W[l], sizeof(float) * nW[l], cudaMemcpyDeviceToDevice, c->stream), "W copy");
      CK(c, cudaMemcpyAsync(c->net + offb[l], b[l], sizeof(float) * nb[l], cudaMemcpyDeviceToDevice, c->stream), "b copy");
    } else {
      CK(c, cudaMemcpyAsync(c->net + offW[l], W[l], sizeof(float) * nW[l], cudaMemcpyHostToDevice, c->stream), "W copy");
      CK(c, cudaMemcpyAsync(c->net + offb[l], b[l], sizeof(float) * nb[l], cudaMemcpyHostToDevice, c->stream), "b copy");
    }
  }
  if (H == kTcHidden) CK(c, tc_pack(c->net, c->tc_img[0], c->tc_img[1], c->stream), "operand image pack");
  c->net_host.resize((size_t)net_floats(H));
  CK(c, cudaMemcpyAsync(c->net_host.data(), c->net, sizeof(float) * c->net_host.size(), cudaMemcpyDeviceToHost,
                        c->stream), "network read-back");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  c->have_net = true;
  return ITMPC_OK;
}

itmpc_status itmpc_set_costmaps(itmpc_ctx *c, int32_t n_maps, const float *const *maps, int32_t width,
                                int32_t height, float res, float origin_x, float origin_y, int32_t on_device) {
  if (!c) return ITMPC_ERR_ARG;
  drop_host_graph(c);
  if (n_maps < 1 || !maps || width < 1 || height < 1 || (int64_t)width * height > (int64_t)1 << 30)
    return fail(c, ITMPC_ERR_ARG, "bad costmap shape %d x %d (x %d)", width, height, n_maps);
  for (int i = 0; i < n_maps; ++i)
    if (!maps[i]) return fail(c, ITMPC_ERR_ARG, "costmap %d is NULL", i);
  if (!(res > 0.f) || !finite(res) || !finite(origin_x) || !finite(origin_y))
    return fail(c, ITMPC_ERR_ARG, "res must be finite and > 0, origin finite");
  const size_t n = (size_t)width * height;
  if (!c->map || (size_t)c->map_w * c->map_h * c->n_maps != n * n_maps) {
    if (c->map) {
      CK(c, cudaStreamSynchronize(c->stream), "sync");
      cudaFree(c->map);
      c->map = nullptr;
      c->have_map = false;
    }
    CK(c, cudaMalloc((void **)&c->map, sizeof(float) * n * n_maps), "costmap cudaMalloc");
  }
  for (int i = 0; i < n_maps; ++i)
    CK(c, cudaMemcpyAsync(c->map + n * i, maps[i], sizeof(float) * n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
       "costmap copy");
  if (!on_device) CK(c, cudaStreamSynchronize(c->stream), "sync");
  c->map_w = width;
  c->map_h = height;
  c->n_maps = n_maps;
  c->res = res;
  c->origin_x = origin_x;
  c->origin_y = origin_y;
  c->have_map = true;
  return ITMPC_OK;
}

itmpc_status itmpc_set_basis(itmpc_ctx *c, const float *theta, int32_t on_device) {
  if (!c) return ITMPC_ERR_ARG;
  if (!theta) return fail(c, ITMPC_ERR_ARG, "theta is NULL");
  if (c->cfg.dynamics != ITMPC_DYN_BASIS) return fail(c, ITMPC_ERR_ARG, "the context was created for the network model");
  std::vector<float> h(100);
  if (on_device) {
    CK(c, cudaMemcpyAsync(h.data(), theta, sizeof(float) * 100, cudaMemcpyDeviceToHost, c->stream), "theta copy");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
  } else {
    memcpy(h.data(), theta, sizeof(float) * 100);
  }
  for (int i = 0; i < 100; ++i)
    if (!finite(h[i])) return fail(c, ITMPC_ERR_ARG, "theta[%d] is not finite", i);
  if (!c->theta_d) CK(c, cudaMalloc((void **)&c->theta_d, sizeof(float) * 100), "cudaMalloc");
  CK(c, cudaMemcpyAsync(c->theta_d, h.data(), sizeof(float) * 100, cudaMemcpyHostToDevice, c->stream), "theta copy");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  c->theta_host = h;
  c->have_theta = true;
  return ITMPC_OK;
}

itmpc_status itmpc_set_costmap(itmpc_ctx *c, const float *map, int32_t width, int32_t height, float res,
                               float origin_x, float origin_y, int32_t on_device) {
  if (!c) return ITMPC_ERR_ARG;
  drop_host_graph(c);
  if (!map) return fail(c, ITMPC_ERR_ARG, "costmap is NULL");
  const float *maps[1] = {map};
  return itmpc_set_costmaps(c, 1, maps, width, height, res, origin_x, origin_y, on_device);
}

itmpc_status itmpc_reserve_batch(itmpc_ctx *c, int32_t max_instances, int64_t max_total_samples) {
  if (!c) return ITMPC_ERR_ARG;
  if (!batch_capable(c->H)) return fail(c, ITMPC_ERR_ARG, "batched iterations need hidden == 32, 64 or 128");
  if (max_instances < 1 || max_total_samples < 1 || max_total_samples > ((int64_t)1 << 31))
    return fail(c, ITMPC_ERR_ARG, "bad batch capacity");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  void *old[] = {c->inst_d, c->units_d, c->batch_partials, c->batch_costs, c->batch_stats, c->unit_counter};
  for (void *b : old)
    if (b) cudaFree(b);
  if (c->inst_h) cudaFreeHost(c->inst_h);
  if (c->units_h) cudaFreeHost(c->units_h);
  c->inst_d = c->inst_h = nullptr;
  c->units_d = c->units_h = nullptr;
  c->batch_partials = c->batch_costs = c->batch_stats = nullptr;
  c->unit_counter = nullptr;
  const int64_t max_units = max_total_samples / min_unit(c->H) + max_instances;
  if (max_units > ((int64_t)1 << 30)) return fail(c, ITMPC_ERR_ARG, "batch too large");
  CK(c, cudaMalloc((void **)&c->inst_d, sizeof(TpsInstance) * max_instances), "batch cudaMalloc");
  CK(c, cudaMalloc((void **)&c->units_d, sizeof(TpsUnit) * max_units), "batch cudaMalloc");
  CK(c, cudaMalloc((void **)&c->batch_partials, sizeof(float) * max_units * partial_len(c->T_max)),
     "batch cudaMalloc");
  CK(c, cudaMalloc((void **)&c->batch_costs, sizeof(float) * max_total_samples), "batch cudaMalloc");
  CK(c, cudaMalloc((void **)&c->batch_stats, sizeof(float) * ITMPC_STATS_LEN * max_instances), "batch cudaMalloc");
  CK(c, cudaMalloc((void **)&c->unit_counter, sizeof(unsigned int)), "batch cudaMalloc");
  CK(c, cudaMallocHost((void **)&c->inst_h, sizeof(TpsInstance) * max_instances), "batch cudaMallocHost");
  CK(c, cudaMallocHost((void **)&c->units_h, sizeof(TpsUnit) * max_units), "batch cudaMallocHost");
  if (!c->staged) CK(c, cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming), "event");
  CK(c, cudaMemsetAsync(c->unit_counter, 0, sizeof(unsigned int), c->stream), "memset");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  c->batch_max_inst = max_instances;
  c->batch_max_units = (int)max_units;
  c->batch_max_samples = max_total_samples;
  return ITMPC_OK;
}

itmpc_status itmpc_iterate_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst) {
  return run_batch(c, n, inst, nullptr, 0);
}

itmpc_status itmpc_autotune_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, int32_t reps,
                                  int32_t *nt_out, int32_t *ctas_out) {
  itmpc_status st = batch_ready(c);
  if (st != ITMPC_OK) return st;
  if (n < 1 || !inst) return fail(c, ITMPC_ERR_ARG, "empty batch");
  if (reps < 1) reps = 3;
  if (c->cfg.precision != ITMPC_FP32 || (c->H != 32 && c->cfg.dynamics != ITMPC_DYN_BASIS)) {
    // fixed shapes: one 128-row MMA tile per unit (tensor cores), or the wide kernels' GEMM tile
    if (nt_out) *nt_out = batch_nt(c);
    if (ctas_out) *ctas_out = 0;
    return ITMPC_OK;
  }
  // run the caller's batch with its outputs redirected to scratch, so nothing the caller owns changes
  int64_t uo_floats = 0;
  for (int i = 0; i < n; ++i) uo_floats += 2 * (int64_t)std::max(inst[i].T, 0);
  float *uo = nullptr;
  CK(c, cudaMalloc((void **)&uo, sizeof(float) * std::max<int64_t>(uo_floats, 1)), "autotune cudaMalloc");
  std::vector<itmpc_instance> q(inst, inst + n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    q[i].U_out = uo + off;
    off += 2 * (int64_t)std::max(inst[i].T, 0);
    q[i].weights = nullptr;
    q[i].costs = nullptr;
    q[i].stats = nullptr;
  }
  const TpsTile cands[] = {{64, 0}, {64, 5}, {128, 0}, {128, 2}, {256, 0}, {256, 1}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TpsTile best = c->tps_tile;
  float best_ms = INFINITY;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  for (const TpsTile &t : cands) {
    if (ce != cudaSuccess) break;
    st = run_batch_tile(c, n, q.data(), nullptr, 0, t);  // warm-up
    if (st != ITMPC_OK) break;
    float tot = 0.f;
    for (int r = 0; r < reps && st == ITMPC_OK; ++r) {
      ce = cudaEventRecord(e0, c->stream);
      if (ce != cudaSuccess) break;
      st = run_batch_tile(c, n, q.data(), nullptr, 0, t);
      if (st != ITMPC_OK) break;
      ce = cudaEventRecord(e1, c->stream);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) break;
      tot += ms;
    }
    if (st != ITMPC_OK || ce != cudaSuccess) break;
    if (tot / reps < best_ms) {
      best_ms = tot / reps;
      best = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  cudaFree(uo);
  if (st != ITMPC_OK) return st;
  if (ce != cudaSuccess) return cuda_fail(c, ce, "autotune timing");
  // the runs leave the status word of their own (scratch) outputs: clear it
  CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "status reset");
  c->tps_tile = best;
  if (nt_out) *nt_out = best.nt;
  if (ctas_out) *ctas_out = best.ctas_per_sm;
  return ITMPC_OK;
}

itmpc_status itmpc_batch_graph_destroy(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->ginst_d) cudaFree(c->ginst_d);
  if (c->gunits_d) cudaFree(c->gunits_d);
  if (c->gloop_d) cudaFree(c->gloop_d);
  c->graph_exec = nullptr;
  c->ginst_d = nullptr;
  c->gunits_d = nullptr;
  c->gloop_d = nullptr;
  return ITMPC_OK;
}

itmpc_status itmpc_batch_graph_create(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, int32_t closed_loop,
                                      int32_t smoothing, int32_t plant) {
  itmpc_status st = batch_ready(c);
  if (st != ITMPC_OK) return st;
  if (closed_loop && (smoothing < 0 || smoothing > 2))
    return fail(c, ITMPC_ERR_ARG, "smoothing %d not one of 0, 1, 2", smoothing);
  if (closed_loop && inst)
    for (int i = 0; i < n; ++i)
      if (inst[i].U_out == inst[i].U) return fail(c, ITMPC_ERR_ARG, "closed loop: instance %d has U_out == U", i);
  st = itmpc_batch_graph_destroy(c);
  if (st != ITMPC_OK) return st;
  const int nt = batch_nt(c);
  std::vector<TpsInstance> ih((size_t)std::max(n, 1));
  std::vector<TpsUnit> uh((size_t)std::max(c->batch_max_units, 1));
  int u = 0;
  st = build_batch(c, n, inst, nt, ih.data(), uh.data(), &u);
  if (st != ITMPC_OK) return st;
  CK(c, cudaMalloc((void **)&c->ginst_d, sizeof(TpsInstance) * n), "graph cudaMalloc");
  CK(c, cudaMalloc((void **)&c->gunits_d, sizeof(TpsUnit) * u), "graph cudaMalloc");
  CK(c, cudaMemcpy(c->ginst_d, ih.data(), sizeof(TpsInstance) * n, cudaMemcpyHostToDevice), "graph copy");
  CK(c, cudaMemcpy(c->gunits_d, uh.data(), sizeof(TpsUnit) * u, cudaMemcpyHostToDevice), "graph copy");
  const TpsShared sh = batch_shared(c, c->ginst_d, c->gunits_d, n, u);
  int T_hi = 1;
  if (closed_loop) {
    std::vector<LoopItem> li((size_t)n);
    for (int i = 0; i < n; ++i) {
      li[i].T = inst[i].T;
      li[i].U_prime = inst[i].U_out;
      li[i].U = const_cast<float *>(inst[i].U);
      li[i].x = plant ? const_cast<float *>(inst[i].x0) : nullptr;
      li[i].u_applied = inst[i].stats ? inst[i].stats + 5 : nullptr;
      T_hi = std::max(T_hi, inst[i].T);
    }
    CK(c, cudaMalloc((void **)&c->gloop_d, sizeof(LoopItem) * n), "graph cudaMalloc");
    CK(c, cudaMemcpy(c->gloop_d, li.data(), sizeof(LoopItem) * n, cudaMemcpyHostToDevice), "graph copy");
  }
  IterParams lp = make_params(c);
  lp.T = T_hi;
  cudaStream_t cap = nullptr;
  CK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = launch_batch(c, sh, c->tps_tile, cap);
    cudaError_t ea = cudaSuccess;
    if (st == ITMPC_OK && closed_loop)
      ea = loop_launch(c->gloop_d, nullptr, n, c->H, c->net, lp, smoothing, plant, nullptr, cap,
                       c->cfg.dynamics == ITMPC_DYN_BASIS ? c->theta_d : nullptr);
    if (st == ITMPC_OK && ea == cudaSuccess) ea = tps_launch_advance(c->ginst_d, n, cap);
    e = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = ea;
  }
  if (e == cudaSuccess && st == ITMPC_OK) e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (st != ITMPC_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
  return ITMPC_OK;
}

itmpc_status itmpc_batch_graph_launch(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  if (!c->graph_exec) return fail(c, ITMPC_ERR_STATE, "itmpc_batch_graph_create has not been called");
  CK(c, cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
  return ITMPC_OK;
}

}  // extern "C"

namespace {

// Validate a batch and write its host descriptors (nt-sample units, longest horizon first).
itmpc_status build_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, int nt, TpsInstance *inst_h,
                         TpsUnit *units_h, int *n_units) {
  if (n < 1 || n > c->batch_max_inst || !inst) return fail(c, ITMPC_ERR_ARG, "n=%d outside [1, %d]", n, c->batch_max_inst);
  int64_t total = 0;
  int units = 0;
  for (int i = 0; i < n; ++i) {
    const itmpc_instance &q = inst[i];
    if (q.K < 1 || q.T < 1 || q.T > c->T_max) return fail(c, ITMPC_ERR_ARG, "instance %d: bad K/T", i);
    if (q.map_index < 0 || q.map_index >= c->n_maps) return fail(c, ITMPC_ERR_ARG, "instance %d: bad map", i);
    if (!q.x0 || !q.U || !q.U_out) return fail(c, ITMPC_ERR_ARG, "instance %d: NULL pointer", i);
    total += q.K;
    units += (q.K + nt - 1) / nt;
  }
  if (total > c->batch_max_samples || units > c->batch_max_units)
    return fail(c, ITMPC_ERR_ARG, "batch exceeds the reserved capacity");
  const itmpc_config &g = c->cfg;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return inst[a].T > inst[b].T; });
  int64_t rec_off = 0, cost_off = 0;
  for (int i = 0; i < n; ++i) {
    const itmpc_instance &q = inst[i];
    TpsInstance &d = inst_h[i];
    d.K = q.K;
    d.T = q.T;
    const double nimp = ceil((1.0 - (double)g.alpha_explore) * (double)q.K);
    d.n_imp = (int)(nimp < 0 ? 0 : (nimp > q.K ? q.K : nimp));
    d.map = q.map_index;
    d.ctr2 = (uint32_t)q.iter;
    d.ctr3 = (uint32_t)((q.iter >> 32) & 0xFFFFu) | (q.instance << 16);
    d.n_units = (q.K + nt - 1) / nt;
    d.rec_off = (int)rec_off;
    rec_off += (int64_t)d.n_units * partial_len(q.T);
    d.x0 = q.x0;
    d.U = q.U;
    d.U_out = q.U_out;
    d.weights = q.weights;
    d.costs = q.costs ? q.costs : c->batch_costs + cost_off;
    d.stats = q.stats ? q.stats : c->batch_stats + (size_t)ITMPC_STATS_LEN * i;
    d.k_base = 0;
    d.rec_out = nullptr;
    cost_off += q.K;
  }
  int u = 0;
  for (int oi = 0; oi < n; ++oi) {
    const int i = order[oi];
    for (int j = 0; j < inst_h[i].n_units; ++j) units_h[u++] = TpsUnit{i, j * nt, j, 0};
  }
  *n_units = u;
  return ITMPC_OK;
}

TpsShared batch_shared(const itmpc_ctx *c, const TpsInstance *inst_d, const TpsUnit *units_d, int n, int n_units) {
  const itmpc_config &g = c->cfg;
  TpsShared sh{};
  sh.key0 = (uint32_t)g.seed;
  sh.key1 = (uint32_t)(g.seed >> 32);
  sh.sigma0 = g.sigma[0];
  sh.sigma1 = g.sigma[1];
  sh.dt = g.dt;
  sh.umin0 = g.u_min[0]; sh.umin1 = g.u_min[1];
  sh.umax0 = g.u_max[0]; sh.umax1 = g.u_max[1];
  sh.w_track = g.cost_w[0]; sh.w_speed = g.cost_w[1]; sh.w_stab = g.cost_w[2]; sh.w_crash = g.cost_w[3];
  sh.v_des = g.v_des;
  sh.crash_cost = g.crash_cost;
  sh.log2_decay = (float)log2((double)g.crash_decay);
  sh.track_thresh = g.track_thresh;
  sh.slip_thresh = g.slip_thresh;
  sh.map_cap = g.map_cap;
  sh.gamma = g.gamma;
  sh.inv_sig2_0 = g.sigma[0] > 0 ? (float)(1.0 / ((double)g.sigma[0] * g.sigma[0])) : 0.f;
  sh.inv_sig2_1 = g.sigma[1] > 0 ? (float)(1.0 / ((double)g.sigma[1] * g.sigma[1])) : 0.f;
  sh.lambda = g.lambda;
  sh.inv_lambda = (float)(1.0 / (double)g.lambda);
  sh.maps = c->map;
  sh.map_w = c->map_w;
  sh.map_h = c->map_h;
  sh.map_stride = (long long)c->map_w * c->map_h;
  sh.inv_res = (float)(1.0 / (double)c->res);
  sh.origin_x = c->origin_x;
  sh.origin_y = c->origin_y;
  sh.inst = inst_d;
  sh.units = units_d;
  sh.n_units = n_units;
  sh.n_inst = n;
  sh.T_max = c->T_max;
  sh.partials = c->batch_partials;
  sh.unit_counter = c->unit_counter;
  sh.status = c->status;
  return sh;
}

// Units of the tensor-core kernels are one 128-row MMA tile; FP32 units follow the tuned tile.
int batch_nt(const itmpc_ctx *c) {
  if (c->cfg.precision != ITMPC_FP32) return kTpsThreads;
  return (c->H == 32 || c->cfg.dynamics == ITMPC_DYN_BASIS) ? c->tps_tile.nt : wide_unit_samples(c->H);
}

bool single_as_batch(const itmpc_ctx *c, bool debug_out) {
  if (!c->inst_d) return false;
  if (c->cfg.dynamics == ITMPC_DYN_BASIS) return true;  // only the thread-per-sample kernels have it
  if (c->H == 32) return !debug_out && c->cfg.K >= kTpsMinK;
  return c->cfg.K >= kWideMinK;  // the wide kernel writes the states (checkpoints) itself
}

itmpc_status launch_batch(itmpc_ctx *c, const TpsShared &sh, TpsTile tile, cudaStream_t s) {
  const itmpc_config &g = c->cfg;
  if (g.precision != ITMPC_FP32) {
    CK(c, tc_launch(sh, c->tc_img[g.precision == ITMPC_FP8 ? 1 : 0], g.precision, g.activation, s),
       "tensor-core launch");
  } else if (g.dynamics == ITMPC_DYN_BASIS) {
    CK(c, tps_launch(sh, nullptr, c->H, g.activation, tile, s, c->theta_host.data()), "batched basis-model launch");
  } else if (c->H == 32) {
    CK(c, tps_launch(sh, c->net_host.data(), c->H, g.activation, tile, s), "batched launch");
  } else {
    CK(c, wide_launch(sh, c->net, c->H, g.activation, s), "batched wide-network launch");
  }
  return ITMPC_OK;
}

itmpc_status batch_ready(itmpc_ctx *c) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (c->cfg.precision != ITMPC_FP32 && c->H != kTcHidden)
    return fail(c, ITMPC_ERR_ARG, "BF16 / FP8 iterations need hidden == %d", kTcHidden);
  if (!c->inst_d) return fail(c, ITMPC_ERR_STATE, "itmpc_reserve_batch has not been called");
  return ITMPC_OK;
}

itmpc_status run_batch_tile(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, float *states, int n_states,
                            TpsTile tile, int states_every, const ShardSpec *shard) {
  itmpc_status st = batch_ready(c);
  if (st != ITMPC_OK) return st;
  const int nt = (c->cfg.precision == ITMPC_FP32 && (c->H == 32 || c->cfg.dynamics == ITMPC_DYN_BASIS))
                     ? tile.nt : batch_nt(c);
  // the previous call's copies out of the staging buffers must have finished
  CK(c, cudaEventSynchronize(c->staged), "event sync");
  int u = 0;
  st = build_batch(c, n, inst, nt, c->inst_h, c->units_h, &u);
  if (st != ITMPC_OK) return st;
  if (shard) {  // a batch of one instance: the shard of a sample-sharded iteration
    c->inst_h[0].k_base = shard->k_base;
    c->inst_h[0].n_imp = shard->n_imp;
    c->inst_h[0].rec_out = shard->rec_out;
    c->inst_h[0].weights = nullptr;
  }
  // one instance on the tensor-core kernels: it travels in the launch's parameters and its
  // units follow from K (no table upload); otherwise the tables are copied to the device
  const bool inline1 = n == 1 && c->cfg.precision != ITMPC_FP32;
  if (!inline1) {
    CK(c, cudaMemcpyAsync(c->inst_d, c->inst_h, sizeof(TpsInstance) * n, cudaMemcpyHostToDevice, c->stream), "copy");
    CK(c, cudaMemcpyAsync(c->units_d, c->units_h, sizeof(TpsUnit) * u, cudaMemcpyHostToDevice, c->stream), "copy");
    CK(c, cudaEventRecord(c->staged, c->stream), "event");
  }
  TpsShared sh = batch_shared(c, c->inst_d, c->units_d, n, u);
  if (inline1) {
    sh.inline_inst = 1;
    sh.inst0 = c->inst_h[0];
  }
  if (n == 1) {
    sh.single_K = c->inst_h[0].K;
    sh.single_weights = c->inst_h[0].weights != nullptr;
  }
  sh.states_out = states;
  sh.n_states = states ? n_states : 0;
  sh.states_every = states_every;
  return launch_batch(c, sh, tile, c->stream);
}

itmpc_status run_batch(itmpc_ctx *c, int32_t n, const itmpc_instance *inst, float *states, int n_states,
                       int states_every, const ShardSpec *shard) {
  if (!c) return ITMPC_ERR_ARG;
  return run_batch_tile(c, n, inst, states, n_states, c->tps_tile, states_every, shard);
}

}  // namespace

extern "C" {

itmpc_status itmpc_iterate(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, float *U_out,
                           float *weights, float *costs) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !U_out) return fail(c, ITMPC_ERR_ARG, "x0, U and U_out must be non-NULL");
  return run_iteration(c, x0, U, iter, U_out, weights, costs, nullptr, 0, nullptr);
}

// The host-pointer iteration without weights / costs on the fused FP32 kernel, as one graph:
// H2D of the input block, the iteration (its Philox index read from that block), D2H of the
// output block.  Captured at the first such call and after any change of parameters or maps.
static itmpc_status host_graph_iterate(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, float *U_out) {
  const int T = c->cfg.T, T_max = c->T_max;
  if (!c->host_exec) {
    IterParams p = make_params(c);
    set_iter(p, 0, c->cfg.instance);
    p.x0 = reinterpret_cast<const float *>(c->dblk_in);
    p.iter_add = reinterpret_cast<const unsigned long long *>(c->dblk_in + 32);
    p.U = reinterpret_cast<const float *>(c->dblk_in + kHinU);
    // U' and the status word go straight to the pinned output block (mapped into the device's
    // address space): no copy node back; the host clears the status word before each launch.
    unsigned char *out_d = nullptr;
    const bool mapped = cudaHostGetDevicePointer((void **)&out_d, c->hblk_out, 0) == cudaSuccess;
    if (!mapped) cudaGetLastError();
    unsigned char *out = mapped ? out_d : c->dblk_out;
    p.U_out = reinterpret_cast<float *>(out);
    p.status = reinterpret_cast<int *>(out + hout_status(T_max));
    c->host_mapped = mapped;
    p.weights = nullptr;
    p.weights_inline = c->cfg.K <= 16384;
    const Fp32Tile tile = fp32_pick_tile(p.K, p.T, p.H, c->smem_optin);
    cudaStream_t cap = nullptr;
    CK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    cudaError_t e = cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {  // cooperative launch first, else the merge tree
      IterParams q = p;
      if (attempt == 1) q.grid_bar = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        cudaError_t ek = cudaSuccess;
        if (!c->host_mapped) ek = cudaMemsetAsync(q.status, 0, sizeof(int), cap);
        if (ek == cudaSuccess)
          ek = cudaMemcpyAsync(c->dblk_in, c->hblk_in, hin_bytes(T_max), cudaMemcpyHostToDevice, cap);
        if (ek == cudaSuccess) ek = fp32_launch_iterate(q, tile, cap);
        if (ek == cudaSuccess && !c->host_mapped)
          ek = cudaMemcpyAsync(c->hblk_out, c->dblk_out, hout_bytes(T_max), cudaMemcpyDeviceToHost, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = ek;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->host_exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) break;
      cudaGetLastError();
      drop_host_graph(c);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-iteration graph capture");
  }
  memcpy(c->hblk_in, x0, sizeof(float) * 7);
  memcpy(c->hblk_in + 32, &iter, sizeof(iter));
  memcpy(c->hblk_in + kHinU, U, sizeof(float) * 2 * (size_t)T);
  if (c->host_mapped) {
    const int zero = 0;
    memcpy(c->hblk_out + hout_status(T_max), &zero, sizeof(int));
  }
  CK(c, cudaGraphLaunch(c->host_exec, c->stream), "graph launch");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  memcpy(U_out, c->hblk_out, sizeof(float) * 2 * (size_t)T);
  int s = 0;
  memcpy(&s, c->hblk_out + hout_status(T_max), sizeof(int));
  if (s == ITMPC_ERR_NONFINITE) return fail(c, ITMPC_ERR_NONFINITE, "every rollout cost was non-finite; U unchanged");
  if (s == ITMPC_ERR_TIMEOUT) {
    CK(c, cudaMemsetAsync(c->counters, 0, sizeof(unsigned int) * c->n_counters, c->stream), "counter reset");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
  }
  if (s != 0) return fail(c, (itmpc_status)s, "device status %d", s);
  return ITMPC_OK;
}

itmpc_status itmpc_iterate_host(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, float *U_out,
                                float *weights, float *costs) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !U_out) return fail(c, ITMPC_ERR_ARG, "x0, U and U_out must be non-NULL");
  for (int i = 0; i < 7; ++i)
    if (!finite(x0[i])) return fail(c, ITMPC_ERR_ARG, "x0[%d] is not finite", i);
  if (!weights && !costs && c->cfg.precision == ITMPC_FP32 && !single_as_batch(c, false))
    return host_graph_iterate(c, x0, U, iter, U_out);
  const int T = c->cfg.T, K = c->cfg.K;
  CK(c, cudaMemcpyAsync(c->x0_d, x0, sizeof(float) * 7, cudaMemcpyHostToDevice, c->stream), "x0 copy");
  CK(c, cudaMemcpyAsync(c->U_d, U, sizeof(float) * 2 * T, cudaMemcpyHostToDevice, c->stream), "U copy");
  st = run_iteration(c, c->x0_d, c->U_d, iter, c->Uout_d, weights ? c->w_d : nullptr, nullptr, nullptr, 0, nullptr);
  if (st != ITMPC_OK) return st;
  CK(c, cudaMemcpyAsync(U_out, c->Uout_d, sizeof(float) * 2 * T, cudaMemcpyDeviceToHost, c->stream), "U_out copy");
  if (weights) CK(c, cudaMemcpyAsync(weights, c->w_d, sizeof(float) * K, cudaMemcpyDeviceToHost, c->stream), "w copy");
  if (costs) CK(c, cudaMemcpyAsync(costs, c->costs, sizeof(float) * K, cudaMemcpyDeviceToHost, c->stream), "S copy");
  return itmpc_read_status(c);
}

itmpc_status itmpc_read_status(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  int s = 0;
  CK(c, cudaMemcpyAsync(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status copy");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  if (s != 0) {
    CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "status reset");
    // a wait that ran out may have left merge counters or the grid barrier half-way
    if (s == ITMPC_ERR_TIMEOUT)
      CK(c, cudaMemsetAsync(c->counters, 0, sizeof(unsigned int) * c->n_counters, c->stream), "counter reset");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    if (s == ITMPC_ERR_NONFINITE) return fail(c, ITMPC_ERR_NONFINITE, "every rollout cost was non-finite; U unchanged");
    return fail(c, (itmpc_status)s, "device status %d", s);
  }
  return ITMPC_OK;
}

itmpc_status itmpc_get_stats(itmpc_ctx *c, float out[ITMPC_STATS_LEN]) {
  if (!c || !out) return ITMPC_ERR_ARG;
  CK(c, cudaMemcpyAsync(out, c->stats, sizeof(float) * ITMPC_STATS_LEN, cudaMemcpyDeviceToHost, c->stream), "stats copy");
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  return ITMPC_OK;
}

itmpc_status itmpc_noise(itmpc_ctx *c, uint64_t iter, float *eps) {
  if (!c) return ITMPC_ERR_ARG;
  if (!eps) return fail(c, ITMPC_ERR_ARG, "eps is NULL");
  if (reinterpret_cast<uintptr_t>(eps) & 7u) return fail(c, ITMPC_ERR_ARG, "eps must be 8-byte aligned");
  IterParams p = make_params(c);
  set_iter(p, iter, c->cfg.instance);
  CK(c, launch_noise(p, eps, c->stream), "noise launch");
  return ITMPC_OK;
}

itmpc_status itmpc_rollout_states(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, int32_t n,
                                  float *states, float *costs) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !states || n < 0 || n > c->cfg.K) return fail(c, ITMPC_ERR_ARG, "bad rollout_states arguments");
  return run_iteration(c, x0, U, iter, c->Uout_d, nullptr, costs, states, n, nullptr);
}

itmpc_status itmpc_philox4x32_10(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int64_t n, void *stream) {
  if (!ctr || !key || !out || n < 0) return ITMPC_ERR_ARG;
  cudaError_t e = launch_philox(ctr, key[0], key[1], out, n, (cudaStream_t)stream);
  if (e != cudaSuccess) { cudaGetLastError(); return ITMPC_ERR_CUDA; }
  return ITMPC_OK;
}

itmpc_status itmpc_tanh_f32(const float *x, float *y, int64_t n, void *stream) {
  if (!x || !y || n < 0) return ITMPC_ERR_ARG;
  cudaError_t e = launch_tanh(x, y, n, (cudaStream_t)stream);
  if (e != cudaSuccess) { cudaGetLastError(); return ITMPC_ERR_CUDA; }
  return ITMPC_OK;
}

itmpc_status itmpc_merge_partials(int32_t n_shards, int32_t T, const float *partials, const float *U, float lambda,
                                  float *U_out) {
  if (n_shards < 1 || T < 1 || !partials || !U || !U_out || !(lambda > 0.f)) return ITMPC_ERR_ARG;
  const int PL = partial_len(T);
  double rho = INFINITY;
  for (int s = 0; s < n_shards; ++s) {
    const double r = partials[(size_t)s * PL];
    if (isfinite(r) && r < rho) rho = r;
  }
  if (!isfinite(rho)) {
    for (int o = 0; o < 2 * T; ++o) U_out[o] = U[o];
    return ITMPC_ERR_NONFINITE;
  }
  double eta = 0.0, eta_imp = 0.0;
  for (int s = 0; s < n_shards; ++s) {
    const float *r = partials + (size_t)s * PL;
    const double sc = isfinite(r[0]) ? exp(-((double)r[0] - rho) / lambda) : 0.0;
    eta += sc * r[1];
    eta_imp += sc * r[2];
  }
  for (int o = 0; o < 2 * T; ++o) {
    double E = 0.0;
    for (int s = 0; s < n_shards; ++s) {
      const float *r = partials + (size_t)s * PL;
      const double sc = isfinite(r[0]) ? exp(-((double)r[0] - rho) / lambda) : 0.0;
      E += sc * r[8 + o];
    }
    U_out[o] = (float)((double)U[o] * (eta_imp / eta) + E / eta);
  }
  return ITMPC_OK;
}

itmpc_status itmpc_iterate_shard(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, int64_t k_base,
                                 int64_t K_total, float *partial, float *costs) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !partial) return fail(c, ITMPC_ERR_ARG, "x0, U and partial must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(partial) & 3u) != 0) return fail(c, ITMPC_ERR_ARG, "partial must be 4-byte aligned");
  const int64_t K = c->cfg.K;
  if (k_base < 0 || K_total < k_base + K || K_total > (int64_t)INT32_MAX)
    return fail(c, ITMPC_ERR_ARG, "need 0 <= k_base, k_base + K <= K_total <= 2^31 - 1 (k_base=%lld K=%lld K_total=%lld)",
                (long long)k_base, (long long)K, (long long)K_total);
  const double nimp = ceil((1.0 - (double)c->cfg.alpha_explore) * (double)K_total);
  ShardSpec sp{};
  sp.k_base = (uint32_t)k_base;
  sp.n_imp = (int)(nimp < 0 ? 0 : (nimp > (double)K_total ? K_total : nimp));
  sp.rec_out = partial;
  return run_iteration(c, x0, U, iter, c->Uout_d, nullptr, costs, nullptr, 0, nullptr, 1, &sp);
}

itmpc_status itmpc_merge_shards(itmpc_ctx *c, int32_t n_shards, const float *partials, int64_t K_total,
                                const float *U, float *U_out, const float *costs, float *weights) {
  if (!c) return ITMPC_ERR_ARG;
  if (n_shards < 1 || !partials || !U || !U_out) return fail(c, ITMPC_ERR_ARG, "n_shards >= 1, partials, U, U_out");
  if (K_total < 1 || K_total > (int64_t)INT32_MAX) return fail(c, ITMPC_ERR_ARG, "K_total outside [1, 2^31 - 1]");
  if (weights && !costs) return fail(c, ITMPC_ERR_ARG, "weights need this device's costs");
  if ((reinterpret_cast<uintptr_t>(partials) & 15u) != 0)
    return fail(c, ITMPC_ERR_ARG, "partials must be 16-byte aligned (records are copied in bulk)");
  IterParams p = make_params(c);
  p.K = (int)K_total;  // the free energy's normalisation
  p.U = U;
  p.U_out = U_out;
  p.costs = const_cast<float *>(costs);
  p.weights = weights;
  p.n_states = costs ? c->cfg.K : 0;
  CK(c, launch_merge_records(p, partials, n_shards, c->stream), "shard merge launch");
  return ITMPC_OK;
}

itmpc_status itmpc_update_from_noise(itmpc_ctx *c, const float *eps, const float *weights, const float *U,
                                     float *U_out) {
  if (!c) return ITMPC_ERR_ARG;
  if (!eps || !weights || !U || !U_out) return fail(c, ITMPC_ERR_ARG, "eps, weights, U and U_out must be non-NULL");
  if (reinterpret_cast<uintptr_t>(eps) & 7u) return fail(c, ITMPC_ERR_ARG, "eps must be 8-byte aligned");
  const IterParams p = make_params(c);
  CK(c, wsum_launch(p.K, p.T, p.n_imp, eps, weights, U, U_out, c->wsum_part, c->sms, c->stream),
     "materialised-noise update launch");
  return ITMPC_OK;
}

itmpc_status itmpc_iterate_cem(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, float delta,
                               float *U_out, float *weights, float *costs) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !U_out) return fail(c, ITMPC_ERR_ARG, "x0, U and U_out must be non-NULL");
  if (!(delta >= 0.0f && delta <= 1.0f)) return fail(c, ITMPC_ERR_ARG, "eliteness threshold %g outside [0, 1]", delta);
  float *S = costs ? costs : c->costs;
  st = run_iteration(c, x0, U, iter, c->Uout_d, nullptr, S, nullptr, 0, nullptr);
  if (st != ITMPC_OK) return st;
  IterParams p = make_params(c);
  set_iter(p, iter, c->cfg.instance);
  p.U = U;
  p.U_out = U_out;
  const int zeta0 = (int)floor((double)c->cfg.K * (1.0 - (double)delta) + 0.5);
  CK(c, cem_launch(p, zeta0, S, weights ? weights : c->w_d, c->cem_scal, c->stream), "cross-entropy launch");
  return ITMPC_OK;
}

itmpc_status itmpc_control_step(itmpc_ctx *c, float *x, float *U, uint64_t iter, int32_t smoothing, int32_t plant,
                                float *u_applied) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x || !U) return fail(c, ITMPC_ERR_ARG, "x and U must be non-NULL");
  if (smoothing < 0 || smoothing > 2) return fail(c, ITMPC_ERR_ARG, "smoothing %d not one of 0, 1, 2", smoothing);
  st = run_iteration(c, x, U, iter, c->Uout_d, nullptr, nullptr, nullptr, 0, nullptr);
  if (st != ITMPC_OK) return st;
  const LoopItem it{c->cfg.T, c->Uout_d, U, plant ? x : nullptr, u_applied};
  CK(c, loop_launch(nullptr, &it, 1, c->H, c->net, make_params(c), smoothing, plant, nullptr, c->stream,
                    c->cfg.dynamics == ITMPC_DYN_BASIS ? c->theta_d : nullptr),
     "closed-loop launch");
  return ITMPC_OK;
}

itmpc_status itmpc_control_graph_destroy(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  CK(c, cudaStreamSynchronize(c->stream), "sync");
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  c->loop_exec = nullptr;
  return ITMPC_OK;
}

itmpc_status itmpc_control_graph_create(itmpc_ctx *c, float *x, float *U, uint64_t iter0, int32_t smoothing,
                                        int32_t plant, float *u_applied) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!x || !U) return fail(c, ITMPC_ERR_ARG, "x and U must be non-NULL");
  if (smoothing < 0 || smoothing > 2) return fail(c, ITMPC_ERR_ARG, "smoothing %d not one of 0, 1, 2", smoothing);
  if (c->cfg.precision != ITMPC_FP32 || single_as_batch(c, false))
    return fail(c, ITMPC_ERR_ARG, "this configuration runs as a batch of one: use itmpc_batch_graph_create");
  st = itmpc_control_graph_destroy(c);
  if (st != ITMPC_OK) return st;
  if (!c->loop_ctr) CK(c, cudaMalloc((void **)&c->loop_ctr, sizeof(unsigned long long)), "cudaMalloc");
  CK(c, cudaMemset(c->loop_ctr, 0, sizeof(unsigned long long)), "memset");
  IterParams p = make_params(c);
  set_iter(p, iter0, c->cfg.instance);
  p.x0 = x;
  p.U = U;
  p.U_out = c->Uout_d;
  p.weights = nullptr;
  p.weights_inline = c->cfg.K <= 16384;
  p.iter_add = c->loop_ctr;
  const Fp32Tile tile = fp32_pick_tile(p.K, p.T, p.H, c->smem_optin);
  const LoopItem it{c->cfg.T, c->Uout_d, U, plant ? x : nullptr, u_applied};
  cudaStream_t cap = nullptr;
  CK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
  // first with the cooperative launch (grid barrier, distributed merge) when the device
  // captures it; else the ordinary launch and its merge tree (no grid barrier)
  cudaError_t e = cudaSuccess;
  for (int attempt = 0; attempt < 2; ++attempt) {
    IterParams q = p;
    if (attempt == 1) q.grid_bar = nullptr;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ek = fp32_launch_iterate(q, tile, cap);
      if (ek == cudaSuccess) ek = loop_launch(nullptr, &it, 1, c->H, c->net, q, smoothing, plant, c->loop_ctr, cap);
      e = cudaStreamEndCapture(cap, &graph);
      if (e == cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->loop_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) break;
    cudaGetLastError();
    if (c->loop_exec) {
      cudaGraphExecDestroy(c->loop_exec);
      c->loop_exec = nullptr;
    }
  }
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_fail(c, e, "closed-loop graph capture");
  return ITMPC_OK;
}

itmpc_status itmpc_control_graph_launch(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  if (!c->loop_exec) return fail(c, ITMPC_ERR_STATE, "itmpc_control_graph_create has not been called");
  CK(c, cudaGraphLaunch(c->loop_exec, c->stream), "graph launch");
  return ITMPC_OK;
}

int64_t itmpc_adjoint_ckpt_floats(int32_t K, int32_t T, int32_t every) {
  if (K < 1 || T < 1 || every < 1 || every > ITMPC_ADJ_MAX_EVERY) return -1;
  return (int64_t)K * (T / every + 1) * 7;
}

itmpc_status itmpc_reserve_adjoint(itmpc_ctx *c) {
  if (!c) return ITMPC_ERR_ARG;
  if (c->H != 32 && c->H != 64) return fail(c, ITMPC_ERR_ARG, "the adjoint form needs hidden == 32 or 64 (got %d)", c->H);
  if (c->adj_part) return ITMPC_OK;
  CK(c, cudaMalloc((void **)&c->adj_part, sizeof(float) * adj_part_floats(c->K_cap, c->H, c->T_max)), "cudaMalloc");
  CK(c, cudaMalloc((void **)&c->adj_scal, sizeof(float) * 4), "cudaMalloc");
  return ITMPC_OK;
}

namespace {
itmpc_status adj_check(itmpc_ctx *c, int32_t every) {
  itmpc_status st = ready(c);
  if (st != ITMPC_OK) return st;
  if (!c->adj_part) return fail(c, ITMPC_ERR_STATE, "itmpc_reserve_adjoint has not been called");
  if (c->cfg.precision != ITMPC_FP32) return fail(c, ITMPC_ERR_ARG, "the adjoint form is FP32 only");
  if (c->cfg.dynamics != ITMPC_DYN_NETWORK) return fail(c, ITMPC_ERR_ARG, "the adjoint form needs the network model");
  if (every < 1 || every > ITMPC_ADJ_MAX_EVERY)
    return fail(c, ITMPC_ERR_ARG, "checkpoint interval %d outside [1, %d]", every, ITMPC_ADJ_MAX_EVERY);
  if (adj_plan(c->cfg.K, c->H, every, c->cfg.T, c->sms, c->smem_optin).smem > c->smem_optin)
    return fail(c, ITMPC_ERR_ARG, "checkpoint interval %d with T=%d needs more shared memory than a CTA has", every,
                c->cfg.T);
  return ITMPC_OK;
}
}  // namespace

itmpc_status itmpc_iterate_fwd(itmpc_ctx *c, const float *x0, const float *U, uint64_t iter, int32_t every,
                               float *ckpt, float *U_out, float *weights, float *costs, float *J) {
  itmpc_status st = adj_check(c, every);
  if (st != ITMPC_OK) return st;
  if (!x0 || !U || !ckpt || !U_out || !weights || !costs)
    return fail(c, ITMPC_ERR_ARG, "x0, U, ckpt, U_out, weights and costs must be non-NULL");
  if (U_out == U) return fail(c, ITMPC_ERR_ARG, "U_out may not alias U: the backward pass needs U");
  st = run_iteration(c, x0, U, iter, U_out, weights, costs, ckpt, c->cfg.K, nullptr, every);
  if (st != ITMPC_OK) return st;
  const IterParams p = make_params(c);
  CK(c, adj_launch_scalars(p.K, p.T, p.n_imp, weights, costs, U_out, nullptr, nullptr, c->adj_scal, J, c->stream),
     "adjoint scalars launch");
  return ITMPC_OK;
}

itmpc_status itmpc_iterate_bwd(itmpc_ctx *c, const float *U, uint64_t iter, int32_t every, const float *ckpt,
                               const float *weights, const float *costs, const float *U_out, const float *gJ,
                               const float *gU_out, float *g_cost_w, float *g_U, float *g_net) {
  itmpc_status st = adj_check(c, every);
  if (st != ITMPC_OK) return st;
  if (!U || !ckpt || !weights || !costs || !U_out || !g_cost_w || !g_U || !g_net)
    return fail(c, ITMPC_ERR_ARG, "U, ckpt, weights, costs, U_out and the three gradient outputs must be non-NULL");
  AdjParams a{};
  a.p = make_params(c);
  set_iter(a.p, iter, c->cfg.instance);
  a.p.U = U;
  a.ckpt = ckpt;
  a.every = every;
  a.w = weights;
  a.S = costs;
  a.gUo = gU_out;
  a.scal = c->adj_scal;
  a.part = c->adj_part;
  CK(c, adj_launch_scalars(a.p.K, a.p.T, a.p.n_imp, weights, costs, U_out, gU_out, gJ, c->adj_scal, nullptr,
                           c->stream),
     "adjoint scalars launch");
  const AdjPlan pl = adj_plan(a.p.K, c->H, every, a.p.T, c->sms, c->smem_optin);
  CK(c, adj_launch_backward(a, pl, g_cost_w, g_U, g_net, c->stream), "adjoint backward launch");
  return ITMPC_OK;
}

const char *itmpc_last_error(const itmpc_ctx *c) { return c ? c->err.c_str() : kNoCtx; }

const char *itmpc_status_string(int32_t s) {
  switch (s) {
    case ITMPC_OK: return "ITMPC_OK";
    case ITMPC_ERR_ARG: return "ITMPC_ERR_ARG";
    case ITMPC_ERR_CUDA: return "ITMPC_ERR_CUDA";
    case ITMPC_ERR_NONFINITE: return "ITMPC_ERR_NONFINITE";
    case ITMPC_ERR_TIMEOUT: return "ITMPC_ERR_TIMEOUT";
    case ITMPC_ERR_STATE: return "ITMPC_ERR_STATE";
    case ITMPC_ERR_OOM: return "ITMPC_ERR_OOM";
    default: return "unknown status";
  }
}

int32_t itmpc_version(void) { return 100; }

void itmpc_destroy(itmpc_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"
