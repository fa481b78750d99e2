// itmpc_internal.h -- shared between the C-ABI layer and the kernels (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace itmpc {

// Packed network layout (floats): W1 [H][6], b1 [H], W2 [H][H], b2 [H], W3 [4][H], b3 [4].
__host__ __device__ constexpr int net_off_W1(int) { return 0; }
__host__ __device__ constexpr int net_off_b1(int H) { return 6 * H; }
__host__ __device__ constexpr int net_off_W2(int H) { return 7 * H; }
__host__ __device__ constexpr int net_off_b2(int H) { return 7 * H + H * H; }
__host__ __device__ constexpr int net_off_W3(int H) { return 8 * H + H * H; }
__host__ __device__ constexpr int net_off_b3(int H) { return 12 * H + H * H; }
__host__ __device__ constexpr int net_floats(int H) { return 12 * H + H * H + 4; }

// One partial record per CTA: [rho, eta, eta_imp, sum e^2, n_finite, -, -, -, E[T][2], pad]
// padded to a multiple of 4 floats so every record starts 16-byte aligned.
__host__ __device__ constexpr int partial_len(int T) { return 8 + ((2 * T + 3) & ~3); }

constexpr int ITMPC_MAX_T_DEV = 512;  // equals ITMPC_MAX_T of the public header

// Everything one fused iteration launch needs.  Built on the host per call.
struct IterParams {
  int K, T, n_imp, H;
  int activation;
  // noise: counter words 2 and 3, key words 0 and 1
  uint32_t ctr2, ctr3, key0, key1;
  float sigma0, sigma1;
  // dynamics
  float dt, umin0, umin1, umax0, umax1;
  // cost
  float w_track, w_speed, w_stab, w_crash;
  float v_des, crash_cost, log2_decay, track_thresh, slip_thresh, map_cap;
  float gamma, inv_sig2_0, inv_sig2_1;
  float lambda, inv_lambda;
  // map
  const float *map;
  int map_w, map_h;
  float inv_res, origin_x, origin_y;
  // network (packed, device)
  const float *net;
  // inputs
  const float *x0, *U;
  // outputs and scratch
  float *U_out;
  float *weights;      // may be null
  float *costs;        // never null (context buffer when the caller gives none)
  float *partials;     // n_cta x partial_len(T): one record per CTA
  float *group_rec;    // n_group x partial_len(T): one record per group of CTAs
  unsigned int *counters;  // 1 + n_group arrival counters, zero between launches
  unsigned int *grid_bar;  // 2 words (arrivals, generation) of the grid barrier
  int coop;                // 1: cooperative launch, every CTA resident (grid barrier + distributed merge)
  int group;           // CTAs per first-level merge group
  int stage_floats;    // shared memory (floats) from the end of the U block available to the merge
  float *stats;        // ITMPC_STATS_LEN
  int *status;
  int weights_inline;  // last CTA writes the weights itself
  // debug outputs (null in the hot path)
  float *eps_out;      // K x T x 2
  float *states_out;   // n_states x (T / states_every + 1) x 7: x_t at t = 0, every, 2 every, ...
  int n_states;
  int states_every;    // 1: the whole trajectory; N: the adjoint form's checkpoints every N steps
  // device counter added to the iteration index (a replayed closed-loop graph advances it), or null
  const unsigned long long *iter_add;
  // sample-sharded iteration: local sample k is global sample k_base + k (its Philox counter word 0
  // and its place in the exploration split, n_imp counting global samples); when rec_out is set the
  // final merge writes the merged partial record there instead of U', the weights and the stats
  uint32_t k_base;
  float *rec_out;
};

// Launch shape of the FP32 fused kernel: nwarps warps per CTA, spw samples per
// warp, and `group` CTAs per first-level merge group.
struct Fp32Tile {
  int nwarps;
  int group;
  int spw;
};

// Scratch sizes (in floats / counters) an iteration of K samples and horizon
// T_max needs for any tile the picker may return.
struct Fp32Scratch {
  size_t partial_floats, group_floats, scale_floats, counters;  // scale_floats: reserved, unused
};
Fp32Scratch fp32_scratch(int K, int T_max, int H);

Fp32Tile fp32_pick_tile(int K, int T, int H, size_t smem_limit);
size_t fp32_smem_bytes(int T, int H, Fp32Tile tile);
int fp32_num_ctas(int K, Fp32Tile tile);
cudaError_t fp32_launch_iterate(const IterParams &p, Fp32Tile tile, cudaStream_t s);
cudaError_t launch_finalize_weights(const IterParams &p, cudaStream_t s);
// Merge n partial records (device, stride partial_len(p.T)) on one CTA: U' from p.U into p.U_out
// and the stats (p.K = the samples of all records, for the free energy); then, when p.weights is
// set, the weights of p.n_states local costs p.costs under the merged rho and eta.
cudaError_t launch_merge_records(const IterParams &p, const float *recs, int n, cudaStream_t s);

// ---- thread-per-sample path (many samples: large K, or many instances) ----
constexpr int kTpsThreads = 128;  // samples per work unit of the tensor-core kernels (one MMA tile)
constexpr int kTpsMinUnit = 64;   // smallest FP32 unit: batch buffers are sized for it

// Launch shape of the thread-per-sample FP32 kernel (chosen by itmpc_autotune_batch):
// nt samples (= threads) per unit and CTA; at most ctas_per_sm resident CTAs (0: occupancy limit).
struct TpsTile {
  int nt;
  int ctas_per_sm;
};

// One MPC instance, as the device sees it.
struct TpsInstance {
  int K, T, n_imp, map;
  uint32_t ctr2, ctr3;
  int rec_off;   // float offset of its first partial record
  int n_units;   // its work units = its records (stride partial_len(T))
  const float *x0, *U;
  float *U_out, *weights, *costs, *stats;
  // sample-sharded iteration (as IterParams::k_base / rec_out): global index of sample 0, and the
  // merged record's destination (null: write U', weights and stats)
  uint32_t k_base;
  float *rec_out;
};

// A work unit: nt consecutive samples of one instance (128 for the tensor-core kernels).
struct TpsUnit {
  int inst, k0, idx, pad;  // idx: the unit's index within its instance
};

// Everything the instances share.
struct TpsShared {
  uint32_t key0, key1;
  float sigma0, sigma1, dt, umin0, umin1, umax0, umax1;
  float w_track, w_speed, w_stab, w_crash;
  float v_des, crash_cost, log2_decay, track_thresh, slip_thresh, map_cap;
  float gamma, inv_sig2_0, inv_sig2_1, lambda, inv_lambda;
  const float *maps;
  int map_w, map_h;
  long long map_stride;
  float inv_res, origin_x, origin_y;
  const TpsInstance *inst;
  const TpsUnit *units;
  int n_units, n_inst, T_max, pad;
  float *partials;
  unsigned int *unit_counter;
  int *status;
  // states of samples 0..n_states-1 of instance 0, or null: x_0..x_T (n_states x (T+1) x 7) for the
  // debug outputs; the FP32 wide-network kernel writes x_t at t = 0, e, 2e, ... with e = states_every
  // (n_states x (T/e + 1) x 7: the adjoint form's checkpoints)
  float *states_out;
  int n_states, states_every;
  // a batch of one instance: its K and whether it writes weights (the merge then spreads the
  // weights over several CTAs); 0 otherwise
  int single_K, single_weights;
  // inline_inst = 1: the one instance is inst0 (in the launch's parameters, no table upload) and
  // unit u is its samples 128 u .. 128 u + 127 (the tensor-core kernels and their merge)
  int inline_inst;
  TpsInstance inst0;
};

// Network values in kernel parameter space (constant bank): FMA operands read
// the weights directly.
template <int H>
struct TpsNet {
  float W1[H * 6], b1[H], W2[H * H], b2[H], W3[4 * H], b3[4];
};

// Launch the rollout (persistent over work units) and the per-instance merge.
// theta_host != null: the basis-function model with coefficients theta_host (25 x 4) instead of the network.
cudaError_t tps_launch(const TpsShared &sh, const float *net_host, int H, int activation, TpsTile tile,
                       cudaStream_t s, const float *theta_host = nullptr);
// Advance every instance's Philox iteration index (counter words 2-3, 48 bits) by one:
// the last node of a captured closed-loop graph, so replay r draws iteration iter + r.
cudaError_t tps_launch_advance(TpsInstance *inst, int n, cudaStream_t s);
// The per-instance merge alone (after any kernel that wrote the units' records);
// also resets the unit counter.
cudaError_t tps_merge(const TpsShared &sh, cudaStream_t s);

// ---- tensor-core (BF16 / FP8) rollout of H = 128 networks over the same work units ----
constexpr int kTcHidden = 128;
// Bytes of the packed operand image of one precision (1 = BF16, 2 = FP8 layer 2).
size_t tc_image_bytes(int precision);
// Build both operand images from the packed FP32 network (device).
cudaError_t tc_pack(const float *net, unsigned char *img_bf16, unsigned char *img_fp8, cudaStream_t s);
// Rollout + records (tensor cores), then tps_merge.
cudaError_t tc_launch(const TpsShared &sh, const unsigned char *image, int precision, int activation,
                      cudaStream_t s);
size_t tps_merge_smem_bytes(int max_units_per_instance, int T_max);

// ---- FP32 rollout of the wide networks (H = 64, 128) as a per-step register-tiled GEMM ----
int wide_unit_samples(int H);  // samples per work unit (16 for H = 64, 32 for H = 128)
size_t wide_smem_bytes(int H, int T_max);
// Rollout + records, then tps_merge.  net: the packed FP32 network on the device.
cudaError_t wide_launch(const TpsShared &sh, const float *net, int H, int activation, cudaStream_t s);
cudaError_t launch_noise(const IterParams &p, float *eps, cudaStream_t s);

// ---- closed loop (closed_loop.cu): smoothing, applied control, plant step, warm start ----
struct LoopItem {
  int T;
  const float *U_prime;  // T x 2, the iteration's weighted mean U'
  float *U;              // T x 2 in/out: read as the nominal sequence, written shifted
  float *x;              // 7 in/out (the plant's state), or null
  float *u_applied;      // 2, or null
};
// One CTA per item: U_s = smoothing(U', U) (0 none, 1 SGF(U'), 2 U + SGF(U' - U)), u_applied = U_s[0],
// x <- F(x, g(u_applied)) when plant and x != null (the FP32 network of the context), U <- shift(U_s)
// with U[T-1] = (0, 0); then *counter += 1 when counter != null (one thread, after the items).
// theta != null: the plant is the basis-function model with these coefficients (device, 25 x 4).
cudaError_t loop_launch(const LoopItem *items_dev, const LoopItem *item_host, int n, int H, const float *net,
                        const IterParams &p, int smoothing, int plant, unsigned long long *counter, cudaStream_t s,
                        const float *theta = nullptr);

// ---- cross-entropy weights (cem.cu): Alg. 3 and the elite-mean update ----
// w (K) and scal[0] = Z, scal[1] = elite count from the costs S; then U_out = the mean of the
// elite samples' v (p.U, p.U_out, noise counters of p).  zeta0 = round(K (1 - delta)).
cudaError_t cem_launch(const IterParams &p, int zeta0, const float *S, float *w, float *scal, cudaStream_t s);

// ---- the control law from materialised noise (wsum.cu), the HBM-bound form of the update ----
size_t wsum_part_floats(int T_max, int sms);
cudaError_t wsum_launch(int K, int T, int n_imp, const float *eps, const float *w, const float *U, float *U_out,
                        float *part, int sms, cudaStream_t s);

// ---- adjoint form (iterate_adj.cu): reverse sweep over checkpointed FP32 rollouts ----
struct AdjParams {
  IterParams p;        // dynamics, costs, noise counters, map, network, U
  const float *ckpt;   // K x (T / every + 1) x 7: x_t at t = 0, every, 2 every, ... (forward launch)
  int every;           // checkpoint interval, 1..32
  int sub;             // sub-segment length (from the launch plan)
  const float *w, *S;  // forward weights and costs (K)
  const float *gUo;    // dL/dU' (T x 2) or null
  const float *scal;   // [J, c0 = gU . U', sum of importance weights, gJ] (adj_launch_scalars)
  float *part;         // per-CTA gradient records
};
// Launch shape of the adjoint backward: warps per CTA (one CTA per SM), CTAs, sub-segment
// length and dynamic shared memory.
struct AdjPlan {
  int nw, n_cta, sub;
  size_t smem;
};
AdjPlan adj_plan(int K, int H, int every, int T, int n_sm, size_t smem_max);
size_t adj_part_floats(int K_cap, int H, int T_max);
cudaError_t adj_launch_scalars(int K, int T, int n_imp, const float *w, const float *S, const float *Uo,
                               const float *gUo, const float *gJ, float *scal, float *J_out, cudaStream_t s);
cudaError_t adj_launch_backward(const AdjParams &a, const AdjPlan &pl, float *g_cost_w, float *g_U, float *g_net,
                                cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n, cudaStream_t s);
cudaError_t launch_tanh(const float *x, float *y, int64_t n, cudaStream_t s);

}  // namespace itmpc
