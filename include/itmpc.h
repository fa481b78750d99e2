/*
 * itmpc.h -- C ABI of the GB300 IT-MPC control-iteration library (libitmpc.so).
 *
 * One control iteration of information-theoretic MPC (Williams, Drews,
 * Goldfain, Rehg, Theodorou, "Information Theoretic Model Predictive Control:
 * Theory and Applications to Autonomous Driving", arXiv 1707.02342):
 *   1. draw K noise sequences eps^k ~ N(0, Sigma) of length T  (Alg. 1),
 *   2. roll every perturbed sequence out through x <- F(x, g(v)) with the
 *      network-plus-kinematics vehicle model of Sec. V-B,
 *   3. add the state cost of Sec. V-C after every step (Alg. 1),
 *   4. weight the samples by exp(-(S_k - rho)/lambda)/eta~ (Alg. 2) and
 *      replace the nominal sequence by the weighted mean of the sampled
 *      controls (Sec. III-D, "IT-Controls").
 * Every step runs in hand-written CUDA kernels for sm_103a.  There is no CPU
 * fallback: without a usable GPU the calls return ITMPC_ERR_CUDA.
 *
 * Conventions shared by all entry points:
 *   - Arrays are row-major FP32 unless stated.  State order is
 *     (p_x, p_y, theta, roll, v_x, v_y, theta_dot), control order
 *     (steer, throttle) (Sec. V-B).
 *   - "device pointer" arguments must point to memory of the device that was
 *     current when the context was created; calls taking them are
 *     asynchronous and ordered on the context's stream.
 *   - No entry point keeps a caller pointer after it returns: set_* calls copy.
 *   - Errors never cross the ABI as exceptions: every call returns an
 *     itmpc_status, and itmpc_last_error() gives a message for the last
 *     failing call on a context.  Argument errors are detected before any GPU
 *     work is queued and leave the context unchanged; every entry point that
 *     takes a context returns ITMPC_ERR_ARG for a NULL one.
 *   - Noise is Philox-4x32-10 (Salmon et al., SC'11) with one block per
 *     (k, t): counter = (k, t, iter_lo, (iter_hi & 0xFFFF) | instance << 16),
 *     key = (seed_lo, seed_hi); words 0 and 1 give u_i = ((w_i >> 8) + 1) 2^-24
 *     and Box-Muller gives (z0, z1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1);
 *     eps = (sigma_0 z0, sigma_1 z1).  The paper does not specify its
 *     generator; this layout lets any iteration be regenerated exactly.
 */
#ifndef ITMPC_H
#define ITMPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ITMPC_OK = 0,
  ITMPC_ERR_ARG = -1,       /* invalid argument (shape, pointer, range) */
  ITMPC_ERR_CUDA = -2,      /* CUDA runtime error, including "no device" */
  ITMPC_ERR_NONFINITE = -3, /* every rollout cost was non-finite: U left unchanged */
  ITMPC_ERR_TIMEOUT = -4,   /* a bounded device-side wait ran out */
  ITMPC_ERR_STATE = -5,     /* call out of order (e.g. iterate before set_dynamics) */
  ITMPC_ERR_OOM = -6        /* device allocation failed */
} itmpc_status;

typedef enum { ITMPC_FP32 = 0, ITMPC_BF16 = 1, ITMPC_FP8 = 2 } itmpc_precision;
typedef enum { ITMPC_ACT_TANH = 0, ITMPC_ACT_IDENTITY = 1 } itmpc_activation;
typedef enum { ITMPC_DYN_NETWORK = 0, ITMPC_DYN_BASIS = 1 } itmpc_dynamics;

#define ITMPC_MAX_K (1 << 24)
#define ITMPC_MAX_T 512
#define ITMPC_STATS_LEN 8

/* Iteration parameters (Alg. 1 inputs; Sec. III-E; Sec. V-C).
 *   K, T            samples and horizon; T <= T_max (fixed at create; 0 means T)
 *   hidden          H of the 6 -> H -> H -> 4 dynamics network (32, 64 or 128)
 *   dt              Euler step of Sec. V-B
 *   lambda          inverse temperature of Alg. 2 (> 0)
 *   gamma           control-cost parameter of Sec. III-E; the term
 *                   gamma u_{t-1}' Sigma^-1 v_{t-1} is added to S when gamma != 0
 *   alpha_explore   fraction of samples drawn around zero (Alg. 1's alpha):
 *                   sample k uses v = u + eps iff k < (1 - alpha) K
 *   sigma           standard deviations, Sigma = diag(sigma^2)
 *   u_min, u_max    bounds of the clamp g (Sec. III-E, "Handling Control Constraints")
 *   cost_w          multipliers of (track, speed, stabilizing, impulse) terms
 *   v_des           speed target; crash_cost the impulse size (1e4 in Sec. V-C);
 *   crash_decay     the 0.9 of the time-decayed track impulse (power t = 1..T);
 *   track_thresh    0.99; slip_thresh 0.75; map_cap 2.5 (Sec. V-C)
 *   seed, instance  Philox key and instance tag
 *   precision       ITMPC_FP32: every layer in FP32 on the FMA pipes (hidden 32, 64, 128);
 *                   ITMPC_BF16 / ITMPC_FP8 (hidden == 128 only): the three network
 *                   layers as tcgen05 tensor-core MMAs over 128-sample tiles with
 *                   FP32 accumulation -- BF16 operands, or layer 2 in FP8 E4M3 with a
 *                   power-of-two per-layer scale; noise, kinematics, costs, the
 *                   normaliser and the weighted sums stay FP32
 *   activation      ITMPC_ACT_TANH (the paper's network) or ITMPC_ACT_IDENTITY
 *                   (an affine network, used by closed-form checks)
 *   dynamics        ITMPC_DYN_NETWORK (the network of Sec. V-B, itmpc_set_dynamics) or
 *                   ITMPC_DYN_BASIS (the basis-function model, itmpc_set_basis; FP32,
 *                   thread-per-sample kernels; fixed at create)
 *   stream          cudaStream_t all calls are ordered on (NULL: legacy default) */
typedef struct {
  int32_t K, T, T_max, hidden;
  float dt, lambda, gamma, alpha_explore;
  float sigma[2];
  float u_min[2], u_max[2];
  float cost_w[4];
  float v_des, crash_cost, crash_decay, track_thresh, slip_thresh, map_cap;
  uint64_t seed;
  uint32_t instance;
  int32_t precision;
  int32_t activation;
  int32_t dynamics;
  void *stream;
} itmpc_config;

typedef struct itmpc_ctx itmpc_ctx;

/* Create a context for cfg on the current device.  Allocates all device
 * buffers the iteration needs for K samples and horizon T_max (no allocation
 * happens in itmpc_iterate).  *out receives the context, or NULL on error.
 * Errors: ITMPC_ERR_ARG (bad cfg), ITMPC_ERR_CUDA / ITMPC_ERR_OOM. */
itmpc_status itmpc_create(const itmpc_config *cfg, itmpc_ctx **out);

/* Replace the iteration parameters.  K may not exceed the K given at create,
 * T may not exceed T_max and hidden may not change.  Host-only; takes effect
 * for calls queued afterwards. */
itmpc_status itmpc_set_config(itmpc_ctx *ctx, const itmpc_config *cfg);

/* Set the stream later calls are queued on (a cudaStream_t, NULL = default). */
itmpc_status itmpc_set_stream(itmpc_ctx *ctx, void *stream);

/* Dynamics network f of Sec. V-B ("Neural Network Model"): two hidden layers
 * with tanh and a linear output, f(z) = W3 tanh(W2 tanh(W1 z + b1) + b2) + b3,
 * z = (roll, v_x, v_y, theta_dot, steer, throttle), f = d x_d / dt.
 *   n_layers must be 3; widths = {6, H, H, 4} with H == cfg.hidden;
 *   W[l] is (widths[l+1] x widths[l]) row-major, b[l] has widths[l+1] entries;
 *   on_device != 0: the pointers are device pointers, else host pointers.
 * The weights are copied into the context (synchronously for host input). */
itmpc_status itmpc_set_dynamics(itmpc_ctx *ctx, int32_t n_layers, const int32_t *widths, const float *const *W,
                                const float *const *b, int32_t on_device);

/* Basis-function dynamics model of Sec. V-B ("Basis Function Model") and the
 * paper's appendix: f(x_d, u) = Theta^T phi(x_d, u) with the 25 basis functions
 * listed there (x_d = (roll, v_x, v_y, r), r the yaw rate; u = (steer, throttle);
 * slip angles alpha_f = arctan(v_y/v_x + 0.45 r/v_x - u_delta),
 * alpha_r = arctan(v_y/v_x - 0.35 r/v_x) for v_x > 0.1, else -u_delta and 0).
 *   theta  25 x 4 row-major (basis i, output o); on_device selects device or host input.
 * Requires cfg.dynamics == ITMPC_DYN_BASIS.  Copied into the context. */
itmpc_status itmpc_set_basis(itmpc_ctx *ctx, const float *theta, int32_t on_device);

/* Track costmap h of Sec. V-C: height x width FP32 texels, row-major (row i,
 * column j), texel (i, j) centred at (origin_x + (j + 0.5) res,
 * origin_y + (i + 0.5) res).  Lookups are bilinear with clamp-to-edge
 * addressing, computed in FP32 in software (the paper's hardware texture
 * filter has 8-bit weights).  The map is copied into the context; a new size
 * reallocates it.  on_device selects device or host input. */
itmpc_status itmpc_set_costmap(itmpc_ctx *ctx, const float *map, int32_t width, int32_t height, float res,
                               float origin_x, float origin_y, int32_t on_device);

/* One control iteration (Alg. 1 body up to the update; Alg. 2).
 *   x0      device, 7 floats: start state
 *   U       device, T x 2: nominal controls u_0..u_{T-1}
 *   iter    Philox counter words 2-3 (use the closed-loop step index)
 *   U_out   device, T x 2: sum_k w_k v_{k,t} (= U + sum_k w_k eps_k when alpha = 0);
 *           may alias U
 *   weights device, K, or NULL: w_k of Alg. 2
 *   costs   device, K, or NULL: S_k, including the gamma term
 * Asynchronous.  A device-side condition (every S_k non-finite) copies U to
 * U_out, zeroes the weights and records ITMPC_ERR_NONFINITE, which
 * itmpc_read_status() returns. */
itmpc_status itmpc_iterate(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, float *U_out,
                           float *weights, float *costs);

/* itmpc_iterate on HOST buffers: copies x0 and U to the device, runs the
 * iteration, copies U_out (and weights/costs when non-NULL) back and waits.
 * Returns the device-side status as well (e.g. ITMPC_ERR_NONFINITE).  Without
 * weights and costs, on the fused FP32 kernel (hidden 32 with K < 4096, hidden
 * 64 / 128 with K < 2048), the call replays one CUDA graph the context captures
 * at the first such call and again after itmpc_set_config / set_stream /
 * set_costmap(s): the upload of (x0, iter, U) from a pinned block and the
 * iteration, whose kernel writes (U_out, status) into a mapped pinned block
 * (copied back by the graph where the block cannot be mapped). */
itmpc_status itmpc_iterate_host(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, float *U_out,
                                float *weights, float *costs);

/* Wait for the context's stream and return the device-side status of the
 * last iteration (ITMPC_OK or ITMPC_ERR_NONFINITE), then clear it. */
itmpc_status itmpc_read_status(itmpc_ctx *ctx);

/* Copy the last iteration's diagnostics to host (waits for the stream):
 * out[0] rho = min_k S_k, out[1] eta~ = sum_k exp(-(S_k - rho)/lambda),
 * out[2] effective sample size 1 / sum_k w_k^2, out[3] free energy estimate
 * -lambda log((1/K) sum_k exp(-S_k/lambda)) (Sec. II, "Free-Energy"),
 * out[4] number of finite costs, out[5..7] reserved. */
itmpc_status itmpc_get_stats(itmpc_ctx *ctx, float out[ITMPC_STATS_LEN]);

/* Several costmaps of one size (the batched form's maps), map i at maps[i].
 * Replaces the map set by itmpc_set_costmap (which is the n_maps = 1 case);
 * single-instance iterations use map 0. */
itmpc_status itmpc_set_costmaps(itmpc_ctx *ctx, int32_t n_maps, const float *const *maps, int32_t width,
                                int32_t height, float res, float origin_x, float origin_y, int32_t on_device);

/* One independent MPC problem of a batched iteration.
 * Every instance shares the context's network and parameters (lambda, sigma,
 * costs, seed); it has its own size, costmap, start state and nominal
 * controls.  Pointers are device pointers; weights, costs and stats may be
 * NULL (stats: ITMPC_STATS_LEN floats as itmpc_get_stats). */
typedef struct {
  int32_t K, T;       /* samples and horizon (T <= the context's T_max) */
  int32_t map_index;  /* index into itmpc_set_costmaps */
  uint32_t instance;  /* Philox instance tag (high half of counter word 3) */
  uint64_t iter;      /* Philox counter words 2-3 */
  const float *x0;    /* 7 floats */
  const float *U;     /* T x 2 */
  float *U_out;       /* T x 2, may alias U */
  float *weights;     /* K or NULL */
  float *costs;       /* K or NULL */
  float *stats;       /* ITMPC_STATS_LEN or NULL */
} itmpc_instance;

/* Reserve device memory for batched iterations of up to max_instances
 * instances with at most max_total_samples samples in all (no allocation
 * happens in itmpc_iterate_batch).  Requires hidden == 32, 64 or 128 (BF16 /
 * FP8: 128). */
itmpc_status itmpc_reserve_batch(itmpc_ctx *ctx, int32_t max_instances, int64_t max_total_samples);

/* One control iteration of n independent instances in one launch (Alg. 1 and
 * Alg. 2 per instance): a persistent kernel pulls (instance, sample tile) work
 * units, longest horizon first, then one CTA per instance merges its partial
 * sums.  The rollout kernel follows the network: one thread per sample with
 * the weights in the constant bank (FP32, hidden 32; unit size from
 * itmpc_autotune_batch), a register-tiled GEMM per step over 16 / 32 samples
 * (FP32, hidden 64 / 128), or tcgen05 MMAs over 128 samples (BF16 / FP8).
 * inst is a host array of n descriptors.  Asynchronous; an instance whose
 * costs are all non-finite gets U_out = U and records ITMPC_ERR_NONFINITE. */
itmpc_status itmpc_iterate_batch(itmpc_ctx *ctx, int32_t n, const itmpc_instance *inst);

/* Choose the launch shape of batched FP32 iterations for this batch by timing
 * it: samples per work unit (= threads per CTA) in {64, 128, 256} and the
 * number of resident CTAs per SM (the occupancy limit or half of it); `reps`
 * timed runs per candidate (0: 3).  The runs write to scratch outputs (the
 * caller's U_out, weights, costs and stats are left untouched; x0 and U are
 * only read); later itmpc_iterate_batch calls and graphs use the winner.
 * The tensor-core (BF16 / FP8) kernels and the FP32 kernels of the wider
 * networks have fixed shapes (a unit is one 128-row MMA tile, or 16 / 32
 * samples for H = 64 / 128), reported without timing.  Synchronous.
 * nt_out, ctas_out (may be NULL): the chosen shape (ctas 0 = occupancy limit). */
itmpc_status itmpc_autotune_batch(itmpc_ctx *ctx, int32_t n, const itmpc_instance *inst, int32_t reps,
                                  int32_t *nt_out, int32_t *ctas_out);

/* Control smoothing of Sec. III-E ("Control Smoothing") applied by the closed-loop
 * step: the 5-point quadratic Savitzky-Golay filter (convolution weights
 * (-3, 12, 17, 12, -3)/35, end values replicated at the edges).  The paper's text
 * filters the weighted mean U'; its Alg. 1 adds the filtered weighted noise to U
 * (U + SGF(U' - U)); both readings are offered. */
typedef enum { ITMPC_SMOOTH_NONE = 0, ITMPC_SMOOTH_SGF = 1, ITMPC_SMOOTH_SGF_DELTA = 2 } itmpc_smoothing;

/* Capture one batched iteration of the n instances into a CUDA graph owned by
 * the context: each itmpc_batch_graph_launch replays the rollout and merge
 * launches and then advances every instance's Philox iteration index by one on
 * the device, so replay r (counting from 0 after create) draws the noise of
 * iteration inst[i].iter + r.
 *   closed_loop 0: the replay is an iteration (U_out == U makes each replay start
 *                  from the previous U').
 *   closed_loop 1: after the merge, every instance runs the end of Alg. 1 (as
 *                  itmpc_control_step): U_s = smoothing(U_out, U); the first control
 *                  U_s[0] goes to stats[5..6] (when stats is given) and, when plant
 *                  != 0, through the noise-free model x0 <- F(x0, g(U_s[0])) (x0 is
 *                  then written: it must be writable device memory); then
 *                  U <- (U_s[1..T-1], (0, 0)).  U (also written) must not alias U_out.
 * The graph keeps the descriptors, the parameters, the network and the costmaps
 * as they are at create (the buffers behind the pointers are read and written by
 * every replay); create it again after changing any of them.  A new create
 * replaces the previous graph.
 * Errors: ITMPC_ERR_STATE before itmpc_reserve_batch, ITMPC_ERR_ARG, ITMPC_ERR_CUDA. */
itmpc_status itmpc_batch_graph_create(itmpc_ctx *ctx, int32_t n, const itmpc_instance *inst, int32_t closed_loop,
                                      int32_t smoothing, int32_t plant);

/* Replay the captured graph once on the context's stream (asynchronous). */
itmpc_status itmpc_batch_graph_launch(itmpc_ctx *ctx);

/* Release the captured graph (waits for the context's stream); no-op without one. */
itmpc_status itmpc_batch_graph_destroy(itmpc_ctx *ctx);

/* The control law of Sec. III-D from materialised noise: U_out[t] = sum_k w_k v_{k,t}
 * = U[t] sum_{k < (1 - alpha) K} w_k + sum_k w_k eps[k][t], for K and T of the
 * context's configuration.  eps: device, K x T x 2 (as itmpc_noise writes it),
 * weights: device, K (normalised), U, U_out: device T x 2 (U_out may not alias U).
 * The streamed form of the update for callers that hold their noise in memory
 * (K T 8 bytes read once); the iterations themselves never write eps.  eps must
 * be 8-byte aligned; with even T and a 16-byte aligned eps the rows are read with
 * 16-byte loads.  Deterministic (fixed summation order).  Asynchronous.
 * Errors: ITMPC_ERR_ARG (NULL pointer, U_out == U, eps not 8-byte aligned),
 * ITMPC_ERR_CUDA. */
itmpc_status itmpc_update_from_noise(itmpc_ctx *ctx, const float *eps, const float *weights, const float *U,
                                     float *U_out);

/* One iteration of the paper's comparison controller, cross-entropy MPC: the
 * same rollouts and costs, the weights of Alg. 3 -- zeta = round(K (1 - delta)),
 * Z = the zeta-th smallest finite cost, w_k = 1/|E| on the elite set
 * E = {k : S_k <= Z} (|E| = zeta without ties; the paper prints S_k < Z, which
 * would leave weights summing to (zeta - 1)/zeta) -- and the same control law,
 * U'_t = sum_k w_k v_{k,t}: the mean of the elite controls.  delta in [0, 1]
 * (0.8 in the paper's experiments); x0, U, U_out (may alias U), weights (K or
 * NULL), costs (K or NULL) as itmpc_iterate.  Every cost non-finite: U_out = U,
 * weights 0, device status ITMPC_ERR_NONFINITE.  itmpc_get_stats reports the
 * information-theoretic diagnostics of the same rollouts.  Asynchronous. */
itmpc_status itmpc_iterate_cem(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, float delta,
                               float *U_out, float *weights, float *costs);

/* One closed-loop step of Alg. 1 for the context's instance: the iteration from
 * state x and nominal sequence U (iteration index iter), then
 *   U_s = U' (smoothing 0), SGF(U') (1) or U + SGF(U' - U) (2),
 *   u_applied = U_s[0] ("SendToActuators"; device, 2 floats, or NULL),
 *   x <- F(x, g(U_s[0])) with the context's network, noise-free, when plant != 0
 *        (a simulated plant; with a real vehicle pass plant = 0 and write the next
 *        state estimate into x),
 *   U <- (U_s[1], ..., U_s[T-1], (0, 0))  (warm start; Initialize = (0, 0)).
 * x (7) and U (T x 2) are device buffers, read and written.  Asynchronous. */
itmpc_status itmpc_control_step(itmpc_ctx *ctx, float *x, float *U, uint64_t iter, int32_t smoothing, int32_t plant,
                                float *u_applied);

/* Capture itmpc_control_step (x, U, u_applied as given; iteration index iter0)
 * into a CUDA graph owned by the context; each itmpc_control_graph_launch replays
 * it and advances a device counter, so replay r uses iteration iter0 + r.  For
 * single iterations that run on the fused FP32 kernel (hidden 32 with K < 4096,
 * hidden 64 / 128 with K < 2048); other configurations return ITMPC_ERR_ARG and
 * use itmpc_batch_graph_create with closed_loop = 1.  The graph keeps the
 * parameters, network and costmap as they are at create; a new create replaces
 * the previous graph (and restarts the counter at 0). */
itmpc_status itmpc_control_graph_create(itmpc_ctx *ctx, float *x, float *U, uint64_t iter0, int32_t smoothing,
                                        int32_t plant, float *u_applied);
itmpc_status itmpc_control_graph_launch(itmpc_ctx *ctx);
itmpc_status itmpc_control_graph_destroy(itmpc_ctx *ctx);

/* Diagnostics for stage-wise checks.
 * itmpc_noise: eps of iteration iter for every (k, t), device K x T x 2,
 *   8-byte aligned (ITMPC_ERR_ARG otherwise).
 * itmpc_rollout_states: the full rollout of samples 0..n-1 (device,
 *   n x (T+1) x 7, states x_0..x_T) plus all costs (device, K); n <= K. */
itmpc_status itmpc_noise(itmpc_ctx *ctx, uint64_t iter, float *eps);
itmpc_status itmpc_rollout_states(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, int32_t n,
                                  float *states, float *costs);

/* Raw Philox-4x32-10 blocks: out[i] = Philox(ctr[i], key) for i < n.
 * ctr, out: device, n x 4 uint32; key: host, 2 words.  stream: cudaStream_t. */
itmpc_status itmpc_philox4x32_10(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int64_t n,
                                 void *stream);

/* The rollout's FP32 tanh applied elementwise (device x, y of n floats), for
 * accuracy checks of the kernel's activation against a reference tanh. */
itmpc_status itmpc_tanh_f32(const float *x, float *y, int64_t n, void *stream);

/* Floats per partial record for horizon T: 8 header words plus 2T sums,
 * padded to a multiple of 4 so that every record is 16-byte aligned. */
#define ITMPC_PARTIAL_STRIDE(T) (8 + ((2 * (T) + 3) & ~3))

/* Merge per-shard partial sums of one iteration whose K samples were split
 * into n_shards disjoint sets (e.g. one per GPU).  Host memory only; no GPU
 * needed.  Shard s contributes the record partials[s * ITMPC_PARTIAL_STRIDE(T) ...]:
 *   [0] rho_s = min S over the shard, [1] eta_s = sum exp(-(S - rho_s)/lambda),
 *   [2] the same sum over importance samples only, [3] sum of squared terms,
 *   [4] finite count, [5..7] unused, [8 + 2t + i] sum e * eps_{t,i}.
 * U_out (T x 2, may alias U) = U * eta_imp/eta + E/eta after rescaling every
 * shard by exp(-(rho_s - rho)/lambda), rho = min rho_s (log-sum-exp merge;
 * Alg. 2's shift by the minimum cost, applied per shard and then globally).
 * Returns ITMPC_ERR_NONFINITE (U copied) when no shard has a finite cost. */
itmpc_status itmpc_merge_partials(int32_t n_shards, int32_t T, const float *partials, const float *U,
                                  float lambda, float *U_out);

/* ---- Sample-sharded iteration (one exchange of partial records) ----
 * Alg. 2's weights need rho = min_k S_k and eta~ over all K samples, but both
 * are log-sum-exp reductions: a subset of the samples can be reduced on its own
 * to the partial record above (shifted by the subset's own minimum), and the
 * records of disjoint subsets merge exactly into U' (Alg. 2's shift applied per
 * shard, then across shards).  A K_total-sample iteration can therefore run as
 * several contexts -- one per GPU, or several on one GPU -- each owning a
 * contiguous range of global sample indices, followed by one exchange of
 * ITMPC_PARTIAL_STRIDE(T) floats per shard (e.g. an all-gather) and a merge.
 * Because the noise of sample k is Philox(k, t, iter) of its GLOBAL index, the
 * sharded iteration draws exactly the samples of the unsharded one; its U'
 * differs only by the order of the final sums.
 *
 * itmpc_iterate_shard: the context's K samples are global samples
 * k_base .. k_base + K - 1 of an iteration of K_total samples.
 *   x0, U, iter   as itmpc_iterate (device); every shard passes the same values
 *   k_base        0 <= k_base and k_base + K <= K_total <= 2^31 - 1
 *   K_total       the whole iteration's sample count: the exploration split of
 *                 Alg. 1 (v = u + eps iff k < (1 - alpha) K_total) uses the global index
 *   partial       device, ITMPC_PARTIAL_STRIDE(T) floats, 4-byte aligned: the shard's
 *                 record [rho_s, eta_s, eta_imp_s, sum of squares, finite count, 0, 0, 0,
 *                 E_s[T][2]] (as itmpc_merge_partials reads it)
 *   costs         device K, or NULL: S of the shard's samples (local index)
 * Works for every precision and network width of the context.  Asynchronous.
 * The weights need the global rho and eta~: itmpc_merge_shards gives them.
 *
 * itmpc_merge_shards: merge n_shards records (device, 16-byte aligned, stride
 * ITMPC_PARTIAL_STRIDE(T) for the context's T) on the GPU into U_out (device
 * T x 2, may alias U) and the context's stats (itmpc_get_stats; the free energy
 * uses K_total); when weights is given (device K), also the weights of this
 * context's own samples from their costs (device K, as itmpc_iterate_shard
 * wrote them) under the merged rho and eta~.  No shard with a finite cost:
 * U_out = U, weights 0, device status ITMPC_ERR_NONFINITE.  Asynchronous. */
itmpc_status itmpc_iterate_shard(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, int64_t k_base,
                                 int64_t K_total, float *partial, float *costs);
itmpc_status itmpc_merge_shards(itmpc_ctx *ctx, int32_t n_shards, const float *partials, int64_t K_total,
                                const float *U, float *U_out, const float *costs, float *weights);

/* One FP32 control iteration that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate GPU memory when they iterate -- a real-time control loop
 * that forbids allocation after start-up (cudaMalloc can synchronise the
 * device and has no latency bound), or a plug-in whose host application has
 * already reserved the device memory.  It computes what itmpc_create +
 * itmpc_set_dynamics + itmpc_set_costmap + itmpc_iterate compute, without a
 * context:
 *   cfg      iteration parameters as for itmpc_create (precision FP32);
 *            K <= ITMPC_NOALLOC_MAX_K, T <= ITMPC_NOALLOC_MAX_T, else ITMPC_ERR_ARG
 *   W, b     device pointers of the three network layers, as itmpc_set_dynamics
 *   map ...  device costmap and its placement, as itmpc_set_costmap (not copied)
 *   x0, U, iter, U_out, weights, costs   as itmpc_iterate (device pointers)
 * Scratch comes from one file-scope device array of ITMPC_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library keeps until the process exits.  The
 * first call on a device resolves that array's address on the current device
 * (once per device).  Every call on a device shares the array and finds the
 * previous call's contents there (the call clears what must start at zero):
 * calls whose work overlaps on the GPU (different streams or threads without
 * ordering) race and give wrong results.  The call queues its work on
 * cfg->stream, then copies the device status to the host and synchronises
 * that stream: it blocks until the iteration is done, so it must not be made
 * while cfg->stream is capturing a CUDA graph.  It returns the device-side
 * status (ITMPC_OK, ITMPC_ERR_NONFINITE with U copied to U_out,
 * ITMPC_ERR_TIMEOUT).  The size limits hold on GB300 (227 KB of shared memory
 * per block); on a GPU with less shared memory per block the kernel runs
 * smaller CTAs, needs more scratch per sample, and the largest sizes may be
 * refused with ITMPC_ERR_ARG. */
#define ITMPC_NOALLOC_SCRATCH_BYTES (4u << 20)
#define ITMPC_NOALLOC_MAX_K 8192
#define ITMPC_NOALLOC_MAX_T 256
itmpc_status itmpc_iterate_noalloc(const itmpc_config *cfg, const float *const *W, const float *const *b,
                                   const float *map, int32_t width, int32_t height, float res, float origin_x,
                                   float origin_y, const float *x0, const float *U, uint64_t iter, float *U_out,
                                   float *weights, float *costs);

/* ---- Adjoint form: reverse-mode derivative of one FP32 iteration ----
 * The paper derives no gradient of its controller; these entry points apply
 * the chain rule to Alg. 1 (rollout, running cost), Alg. 2 (weights) and the
 * control law of Sec. III-D with the noise held fixed.  The iteration's
 * outputs are J = sum_k w_k S_k (the expected weighted cost) and U' (T x 2);
 * given cotangents gJ and gU the backward pass returns the gradient of
 * gJ J + sum_t gU_t . U'_t with respect to the four cost multipliers, the
 * nominal sequence U and the network parameters.  The impulse terms of the
 * cost are piecewise constant (no slope), the clamp g passes the slope only
 * inside [u_min, u_max], and a sample whose weight is 0 contributes nothing.
 * The forward pass stores the rollout states every `every` steps; the
 * backward pass re-runs each segment from its checkpoint, so memory is
 * K x (T / every + 1) x 7 floats instead of the whole trajectory. */
#define ITMPC_ADJ_MAX_EVERY 32

/* Floats of the checkpoint buffer for K samples, horizon T and interval every
 * (K x (T / every + 1) x 7: states x_t at t = 0, every, 2 every, ...), or -1
 * for arguments out of range (every outside [1, ITMPC_ADJ_MAX_EVERY]). */
int64_t itmpc_adjoint_ckpt_floats(int32_t K, int32_t T, int32_t every);

/* Allocate the backward pass's device scratch for the context's K and T_max
 * (per-CTA gradient records).  Requires hidden == 32 or 64 and FP32.
 * Idempotent.  Errors: ITMPC_ERR_ARG, ITMPC_ERR_OOM. */
itmpc_status itmpc_reserve_adjoint(itmpc_ctx *ctx);

/* Forward pass: itmpc_iterate plus checkpoints and J.
 *   x0, U, iter     as itmpc_iterate (device)
 *   every           checkpoint interval (1..ITMPC_ADJ_MAX_EVERY; the shared memory
 *                   of the backward pass must fit, else ITMPC_ERR_ARG)
 *   ckpt            device, itmpc_adjoint_ckpt_floats(K, T, every) floats (written)
 *   U_out           device T x 2 (may NOT alias U), weights and costs device K (written)
 *   J               device, 1 float or NULL: sum_k w_k S_k
 * Asynchronous on the context's stream.  ITMPC_ERR_STATE before itmpc_reserve_adjoint. */
itmpc_status itmpc_iterate_fwd(itmpc_ctx *ctx, const float *x0, const float *U, uint64_t iter, int32_t every,
                               float *ckpt, float *U_out, float *weights, float *costs, float *J);

/* Backward pass for the outputs of an itmpc_iterate_fwd with the same U, iter,
 * every and context parameters (ckpt, weights, costs, U_out are its outputs,
 * unchanged; device).
 *   gJ        device, 1 float, or NULL for 0: dL/dJ
 *   gU_out    device T x 2, or NULL for 0: dL/dU'
 *   g_cost_w  device, 4 floats (written): dL/d cost_w
 *   g_U       device T x 2 (written): dL/dU
 *   g_net     device, 12 H + H^2 + 4 floats (written): dL/d(W1, b1, W2, b2, W3, b3),
 *             packed in that order, W row-major (fan_out x fan_in) as itmpc_set_dynamics
 * The result is deterministic (fixed summation order).  Asynchronous. */
itmpc_status itmpc_iterate_bwd(itmpc_ctx *ctx, const float *U, uint64_t iter, int32_t every, const float *ckpt,
                               const float *weights, const float *costs, const float *U_out, const float *gJ,
                               const float *gU_out, float *g_cost_w, float *g_U, float *g_net);

/* Message for the last failing call on ctx (never NULL). */
const char *itmpc_last_error(const itmpc_ctx *ctx);

/* Name of a status code. */
const char *itmpc_status_string(int32_t status);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t itmpc_version(void);

/* Release every resource of the context (waits for its stream). NULL is a no-op. */
void itmpc_destroy(itmpc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ITMPC_H */
