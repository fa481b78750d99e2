/*
 * itmpc_oracle.c -- plain FP64 CPU oracle of one IT-MPC control iteration.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This file exists only to check the
 * CUDA library against the paper.  The test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg are the only things that may load it.
 * It shares no source, header, table or helper with the CUDA library, and it
 * never calls it.
 *
 * Paper: G. Williams, P. Drews, B. Goldfain, J. M. Rehg, E. A. Theodorou,
 * "Information Theoretic Model Predictive Control: Theory and Applications to
 * Autonomous Driving", arXiv 1707.02342.
 *
 * Everything below is double precision and follows the paper's order of
 * operations without blocking, fusion or reordering:
 *   - Alg. 1 (Sampling Based MPC): draw noise, roll every sample out for T
 *     steps through F(x, g(v)), add the running cost after each step;
 *   - Alg. 2 (Information Theoretic Weight Computation): rho = min_k S_k,
 *     eta~ = sum_k exp(-(S_k - rho)/lambda), w_k = exp(-(S_k - rho)/lambda)/eta~;
 *   - the control law of Sec. III-D (IT-Controls), u_t = sum_k w_k v_{k,t};
 *   - dynamics of Sec. V-B (kinematics k(x) plus a network f(x_d, v));
 *   - the state cost of Sec. V-C (track, speed and stabilizing terms).
 * Where the paper is silent or garbled, the reading taken is stated at the
 * function that implements it.
 *
 * Noise: the paper does not say how its Gaussian samples are produced.  Both
 * this oracle and the CUDA path implement Philox-4x32-10 from its published
 * definition (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
 * Random Numbers: As Easy as 1, 2, 3", SC'11) and the Box-Muller transform
 * (G. E. P. Box, M. E. Muller, Ann. Math. Stat. 29, 1958) independently, so
 * any iteration's noise can be regenerated here exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_NONFINITE (-3)

/* Problem description.  The network weights follow the layout (fan_out x
 * fan_in), row-major: W1 is H x 6, W2 is H x H, W3 is 4 x H. */
typedef struct {
  int32_t K, T, H, activation; /* activation: 0 = tanh, 1 = identity */
  double dt, lambda, gamma, alpha_explore;
  double sigma[2], u_min[2], u_max[2];
  double cost_w[4]; /* multipliers of: track, speed, stabilizing, crash impulses */
  double v_des, crash_cost, crash_decay, track_thresh, slip_thresh, map_cap;
  uint64_t seed;
  uint32_t instance;
  int32_t n_threads;
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  const float *map;
  int32_t map_w, map_h;
  double res, origin_x, origin_y;
  int32_t model;        /* 0: the network of Sec. V-B; 1: the basis-function model (Sec. V-B, appendix) */
  const double *theta;  /* model 1: Theta, 25 x 4 row-major (basis i, output o) */
} oracle_problem;

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon et al., SC'11, Sec. 5): ten rounds of two 32x32->64
 * multiplications with the round constants 0xD2511F53 and 0xCD9E8D57; the
 * key is bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between
 * rounds.                                                                    */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out) {
  for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Uniform in (0, 1]: the top 24 bits of a word, plus one, times 2^-24.  Every
 * such value is exact in binary32 and binary64, so both sides see the same u. */
static double u01(uint32_t a) { return ((double)(a >> 8) + 1.0) * (1.0 / 16777216.0); }

/* Box-Muller: two standard normals from two uniforms. */
void oracle_box_muller(uint32_t a0, uint32_t a1, double z[2]) {
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = u01(a0), u1 = u01(a1);
  double r = sqrt(-2.0 * log(u0));
  z[0] = r * cos(two_pi * u1);
  z[1] = r * sin(two_pi * u1);
}

/* eps^k_t ~ N(0, Sigma), Sigma = diag(sigma_1^2, sigma_2^2) (Sec. II; Alg. 1
 * "Sample E^k").  One Philox block per (k, t):
 *   counter = (k, t, iter_lo, (iter_hi & 0xFFFF) | instance << 16),
 *   key     = (seed_lo, seed_hi);
 * words 0 and 1 feed Box-Muller; words 2 and 3 are unused.                   */
void oracle_noise(const oracle_problem *P, uint64_t iter, int64_t k, int32_t t, double eps[2]) {
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)t, (uint32_t)iter,
                     (uint32_t)((iter >> 32) & 0xFFFFu) | (P->instance << 16)};
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
  uint32_t w[4];
  double z[2];
  oracle_philox4x32_10(ctr, key, w);
  oracle_box_muller(w[0], w[1], z);
  eps[0] = P->sigma[0] * z[0];
  eps[1] = P->sigma[1] * z[1];
}

void oracle_noise_all(const oracle_problem *P, uint64_t iter, double *eps /* K x T x 2 */) {
  for (int64_t k = 0; k < P->K; ++k)
    for (int32_t t = 0; t < P->T; ++t) oracle_noise(P, iter, k, t, eps + 2 * ((size_t)k * P->T + t));
}

/* ------------------------------------------------------------------------- */
/* Sec. V-B, "Neural Network Model": two fully connected hidden layers with
 * hyperbolic-tangent non-linearities and a linear output layer.  Input
 * z = (roll, v_x, v_y, theta_dot, steer, throttle); output = f(x_d, v), the
 * time derivative of x_d = (roll, v_x, v_y, theta_dot).                       */
static double act(const oracle_problem *P, double a) { return P->activation == 1 ? a : tanh(a); }

#define ORACLE_MAX_H 1024

void oracle_mlp(const oracle_problem *P, const double z[6], double d[4]) {
  const int H = P->H;
  double h1[ORACLE_MAX_H], h2[ORACLE_MAX_H];
  for (int j = 0; j < H; ++j) {
    double a = P->b1[j];
    for (int i = 0; i < 6; ++i) a += P->W1[j * 6 + i] * z[i];
    h1[j] = act(P, a);
  }
  for (int j = 0; j < H; ++j) {
    double a = P->b2[j];
    for (int i = 0; i < H; ++i) a += P->W2[(size_t)j * H + i] * h1[i];
    h2[j] = act(P, a);
  }
  for (int o = 0; o < 4; ++o) {
    double a = P->b3[o];
    for (int i = 0; i < H; ++i) a += P->W3[(size_t)o * H + i] * h2[i];
    d[o] = a;
  }
}

/* Sec. V-B, "Basis Function Model", and the paper's appendix: f(x_d, u) =
 * Theta^T phi(x_d, u) with the 25 basis functions listed there, for
 * x_d = (roll, v_x, v_y, r) (r the yaw rate) and u = (u_delta, u_F) =
 * (steer, throttle).  The slip angles are
 *   alpha_f = arctan(v_y/v_x + 0.45 r/v_x - u_delta) if v_x > 0.1, else -u_delta,
 *   alpha_r = arctan(v_y/v_x - 0.35 r/v_x)           if v_x > 0.1, else 0,
 * and "||.||" in the list is read as the absolute value.                    */
void oracle_basis_phi(const double xd[4], const double g[2], double phi[25]) {
  const double th = xd[0], vx = xd[1], vy = xd[2], r = xd[3];
  const double ud = g[0], uF = g[1];
  const int fast = vx > 0.1;
  const double af = fast ? atan(vy / vx + 0.45 * r / vx - ud) : -ud;
  const double ar = fast ? atan(vy / vx - 0.35 * r / vx) : 0.0;
  const double tf = tan(af), tr = tan(ar), sd = sin(ud);
  phi[0] = uF;
  phi[1] = vx / 10.0;
  phi[2] = sd * tf / 1200.0;
  phi[3] = sd * tf * fabs(tf) / (1200.0 * 1200.0);
  phi[4] = sd * tf * tf * tf / (1200.0 * 1200.0 * 1200.0);
  phi[5] = r * vy / 25.0;
  phi[6] = r / 10.0;
  phi[7] = vy / 10.0;
  phi[8] = sd;
  phi[9] = fast ? (vy / vx) / 40.0 : 0.0;
  phi[10] = tf / 1400.0;
  phi[11] = tf * fabs(tf) / (1400.0 * 1400.0);
  phi[12] = tf * tf * tf / (1400.0 * 1400.0 * 1400.0);
  phi[13] = tr / 40.0;
  phi[14] = tr * fabs(tr) / (40.0 * 40.0);
  phi[15] = tr * tr * tr / (40.0 * 40.0 * 40.0);
  phi[16] = r * vx / 50.0;
  phi[17] = th;
  phi[18] = th * r;
  phi[19] = th * vx / 3.0;
  phi[20] = th * vx * r / 5.0;
  phi[21] = vx * vx / 100.0;
  phi[22] = vx * vx * vx / 1000.0;
  phi[23] = uF * uF;
  phi[24] = uF * uF * uF;
}

/* f = Theta^T phi for the input z = (x_d, g(v)). */
void oracle_basis_f(const oracle_problem *P, const double z[6], double d[4]) {
  double phi[25];
  oracle_basis_phi(z, z + 4, phi);
  for (int o = 0; o < 4; ++o) {
    double a = 0.0;
    for (int i = 0; i < 25; ++i) a += P->theta[i * 4 + o] * phi[i];
    d[o] = a;
  }
}

/* g(v): clamp each control into [u_min, u_max] (Sec. III-E, "Handling Control
 * Constraints").  The paper gives no limits; callers pass them. */
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* One explicit-Euler step of the full equations of motion (Sec. V-B):
 *   x_k(t+1) = x_k(t) + k(x(t)) dt,  k(x) = (cos th v_x - sin th v_y,
 *                                            sin th v_x + cos th v_y, th_dot)
 *   x_d(t+1) = x_d(t) + f(x_d(t), v(t)) dt
 * Both halves use the old state x(t).  gv is the already clamped control. */
void oracle_dynamics_step(const oracle_problem *P, const double x[7], const double gv[2], double xn[7]) {
  double th = x[2], vx = x[4], vy = x[5], thd = x[6];
  double z[6] = {x[3], x[4], x[5], x[6], gv[0], gv[1]};
  double f[4];
  if (P->model == 1) oracle_basis_f(P, z, f);
  else oracle_mlp(P, z, f);
  xn[0] = x[0] + (cos(th) * vx - sin(th) * vy) * P->dt;
  xn[1] = x[1] + (sin(th) * vx + cos(th) * vy) * P->dt;
  xn[2] = x[2] + thd * P->dt;
  for (int i = 0; i < 4; ++i) xn[3 + i] = x[3 + i] + f[i] * P->dt;
}

/* Noise-free plant step F(x, g(u)) used by a closed loop (Alg. 1,
 * "SendToActuators"). */
void oracle_plant_step(const oracle_problem *P, const double x[7], const double u[2], double xn[7]) {
  double gv[2] = {clampd(u[0], P->u_min[0], P->u_max[0]), clampd(u[1], P->u_min[1], P->u_max[1])};
  oracle_dynamics_step(P, x, gv, xn);
}

/* h(p_x, p_y): the costmap lookup of Sec. V-C ("Track Cost").  The paper uses
 * the hardware-interpolated texture fetch; this is bilinear interpolation
 * with texel (i, j) centred at (origin_x + (j + 1/2) res, origin_y + (i + 1/2) res)
 * and clamp-to-edge addressing, in double precision. */
static long clamp_index(double i, long n) { return i < 0.0 ? 0 : (i > (double)(n - 1) ? n - 1 : (long)i); }

double oracle_costmap(const oracle_problem *P, double px, double py) {
  double fx = (px - P->origin_x) / P->res - 0.5;
  double fy = (py - P->origin_y) / P->res - 0.5;
  if (isnan(fx) || isnan(fy)) return NAN;
  double jf = floor(fx), if_ = floor(fy);
  double a = fx - jf, b = fy - if_;
  long W = P->map_w, Hh = P->map_h;
  long j0 = clamp_index(jf, W), j1 = clamp_index(jf + 1.0, W);
  long i0 = clamp_index(if_, Hh), i1 = clamp_index(if_ + 1.0, Hh);
  double m00 = P->map[i0 * W + j0], m01 = P->map[i0 * W + j1];
  double m10 = P->map[i1 * W + j0], m11 = P->map[i1 * W + j1];
  return (1.0 - a) * (1.0 - b) * m00 + a * (1.0 - b) * m01 + (1.0 - a) * b * m10 + a * b * m11;
}

/* State cost c(x_t) at loop index t = 1..T (Sec. V-C):
 *   alpha_1 Track + alpha_2 Speed + alpha_3 Stabilizing, with
 *   Track       = h + decay^t * crash * I{h > track_thresh}, h capped at map_cap,
 *   Speed       = (v_x - v_des)^2,
 *   Stabilizing = zeta^2 + crash * I{|zeta| > slip_thresh},
 *   zeta        = -arctan(v_y / |v_x|), read as -atan2(v_y, |v_x|) so that it
 *                 is defined at v_x = 0.
 * The paper prints alpha_1..3 without values.  cost_w[0..2] are those
 * multipliers and cost_w[3] multiplies both impulse terms, so
 *   c = w0 h + w1 Speed + w2 zeta^2 + w3 crash (decay^t I{h>.} + I{|zeta|>.}).
 * comp (optional) receives the four unweighted terms; margin (optional)
 * receives the distance of h and |zeta| to their thresholds.               */
double oracle_state_cost(const oracle_problem *P, const double x[7], int32_t t, double comp[4], double *margin) {
  double h = oracle_costmap(P, x[0], x[1]);
  if (h > P->map_cap) h = P->map_cap;
  double vx = x[4], vy = x[5];
  double zeta = -atan2(vy, fabs(vx));
  double speed = (vx - P->v_des) * (vx - P->v_des);
  double imp = 0.0;
  if (h > P->track_thresh) imp += pow(P->crash_decay, (double)t) * P->crash_cost;
  if (fabs(zeta) > P->slip_thresh) imp += P->crash_cost;
  if (comp) {
    comp[0] = h;
    comp[1] = speed;
    comp[2] = zeta * zeta;
    comp[3] = imp;
  }
  if (margin) {
    double m1 = fabs(h - P->track_thresh), m2 = fabs(fabs(zeta) - P->slip_thresh);
    *margin = m1 < m2 ? m1 : m2;
  }
  return P->cost_w[0] * h + P->cost_w[1] * speed + P->cost_w[2] * zeta * zeta + P->cost_w[3] * imp;
}

/* Alg. 1, inner loop, for one sample k:
 *   x <- x0
 *   for t = 1..T:
 *     v_{t-1} = u_{t-1} + eps_{t-1}  if k < (1 - alpha) K, else eps_{t-1}
 *     x <- F(x, g(v_{t-1}))
 *     S += c(x) + gamma u_{t-1}^T Sigma^{-1} v_{t-1}
 *   S += phi(x)
 * Readings: the control-cost line of Alg. 1 prints v_t inside a loop whose
 * other lines use t-1; v_{t-1} is taken.  The term is skipped when gamma is 0
 * (so that Sigma = 0 stays defined).  phi is not given by the paper and is 0.
 * traj (optional) receives x_0..x_T, (T+1) x 7; comp (optional) receives the
 * five unweighted sums (track, speed, stabilizing, impulses, control term
 * without gamma); margin (optional) the smallest threshold distance along
 * the rollout.  Returns S_k.                                                */
double oracle_rollout_sample(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter,
                             int64_t k, double *traj, double comp[5], double *margin) {
  double x[7], xn[7];
  memcpy(x, x0, sizeof(x));
  if (traj) memcpy(traj, x0, sizeof(x));
  int importance = (double)k < (1.0 - P->alpha_explore) * (double)P->K;
  double S = 0.0, mmin = INFINITY;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int32_t t = 1; t <= P->T; ++t) {
    double eps[2], v[2], gv[2];
    oracle_noise(P, iter, k, t - 1, eps);
    for (int i = 0; i < 2; ++i) {
      v[i] = importance ? U[2 * (t - 1) + i] + eps[i] : eps[i];
      gv[i] = clampd(v[i], P->u_min[i], P->u_max[i]);
    }
    oracle_dynamics_step(P, x, gv, xn);
    memcpy(x, xn, sizeof(x));
    if (traj) memcpy(traj + 7 * (size_t)t, x, sizeof(x));
    double c4[4], m;
    double c = oracle_state_cost(P, x, t, c4, &m);
    if (m < mmin) mmin = m;
    for (int i = 0; i < 4; ++i) acc[i] += c4[i];
    double ctrl = 0.0;
    if (P->gamma != 0.0) {
      ctrl = U[2 * (t - 1)] * v[0] / (P->sigma[0] * P->sigma[0]) +
             U[2 * (t - 1) + 1] * v[1] / (P->sigma[1] * P->sigma[1]);
      acc[4] += ctrl;
    }
    S += c + P->gamma * ctrl;
  }
  if (comp) memcpy(comp, acc, sizeof(acc));
  if (margin) *margin = mmin;
  return S;
}

/* Alg. 2.  Non-finite costs get weight 0 (they stand for rollouts that left
 * the representable range); if no cost is finite the iteration is rejected.
 * The paper's line w_k <- exp(.)/eta uses eta~, the sum it has just formed. */
int oracle_weights(int64_t K, const double *S, double lambda, double *w, double *rho_out, double *eta_out) {
  if (K <= 0 || !(lambda > 0.0)) return ORACLE_ERR_ARG;
  double rho = INFINITY;
  for (int64_t k = 0; k < K; ++k)
    if (isfinite(S[k]) && S[k] < rho) rho = S[k];
  if (!isfinite(rho)) return ORACLE_ERR_NONFINITE;
  double eta = 0.0;
  for (int64_t k = 0; k < K; ++k) eta += isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 0.0;
  for (int64_t k = 0; k < K; ++k) w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) / eta : 0.0;
  if (rho_out) *rho_out = rho;
  if (eta_out) *eta_out = eta;
  return ORACLE_OK;
}

/* Control update.  Sec. III-D (IT-Controls) sets u_t = sum_k w_k v_{k,t}, the
 * weighted mean of the sampled (unclamped) controls.  With alpha = 0 this is
 * Alg. 1's U + sum_k w_k eps_k (the weights sum to one); with exploration
 * samples (v = eps) the two forms differ and the equation's form is taken.
 * Savitzky-Golay smoothing is not applied here.                              */
void oracle_update(const oracle_problem *P, uint64_t iter, const double *w, const double *U, double *U_out) {
  for (int32_t t = 0; t < P->T; ++t) {
    double s0 = 0.0, s1 = 0.0;
    for (int64_t k = 0; k < P->K; ++k) {
      if (w[k] == 0.0) continue;
      double eps[2];
      oracle_noise(P, iter, k, t, eps);
      int importance = (double)k < (1.0 - P->alpha_explore) * (double)P->K;
      double v0 = importance ? U[2 * t] + eps[0] : eps[0];
      double v1 = importance ? U[2 * t + 1] + eps[1] : eps[1];
      s0 += w[k] * v0;
      s1 += w[k] * v1;
    }
    U_out[2 * t] = s0;
    U_out[2 * t + 1] = s1;
  }
}

static int check_problem(const oracle_problem *P) {
  if (!P || P->K <= 0 || P->T <= 0) return ORACLE_ERR_ARG;
  if (P->model == 1) {
    if (!P->theta) return ORACLE_ERR_ARG;
  } else {
    if (P->H <= 0 || P->H > ORACLE_MAX_H) return ORACLE_ERR_ARG;
    if (!P->W1 || !P->b1 || !P->W2 || !P->b2 || !P->W3 || !P->b3) return ORACLE_ERR_ARG;
  }
  if (!P->map || P->map_w <= 0 || P->map_h <= 0 || !(P->res > 0.0)) return ORACLE_ERR_ARG;
  if (!(P->lambda > 0.0)) return ORACLE_ERR_ARG;
  return ORACLE_OK;
}

/* Costs of a list of samples (for sampled parity at large K and for timing).
 * Samples are independent (Alg. 1's loop over k), so they may run on several
 * threads; each sample's arithmetic is unchanged.                           */
int oracle_rollout_many(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter, int64_t n,
                        const int64_t *ks, double *S, double *margins, double *comps /* n x 5 or NULL */) {
  int rc = check_problem(P);
  if (rc) return rc;
  int nt = P->n_threads > 0 ? P->n_threads : 1;
  (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i)
    S[i] = oracle_rollout_sample(P, x0, U, iter, ks[i], NULL, comps ? comps + 5 * i : NULL,
                                 margins ? margins + i : NULL);
  return ORACLE_OK;
}

/* One control iteration: the body of Alg. 1's outer loop up to the update.
 * Outputs U_out (T x 2), weights w (K) and costs S (K).                     */
int oracle_iterate(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter, double *U_out,
                   double *w, double *S) {
  int rc = check_problem(P);
  if (rc) return rc;
  int nt = P->n_threads > 0 ? P->n_threads : 1;
  (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
  for (int64_t k = 0; k < P->K; ++k) S[k] = oracle_rollout_sample(P, x0, U, iter, k, NULL, NULL, NULL);
  rc = oracle_weights(P->K, S, P->lambda, w, NULL, NULL);
  if (rc) return rc;
  oracle_update(P, iter, w, U, U_out);
  return ORACLE_OK;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ========================================================================= */
/* Reverse-mode derivative of one iteration (the adjoint form).
 *
 * The paper derives no gradient of its controller; this is the chain rule
 * applied by hand, in FP64, to the functions above, with the noise held fixed
 * (eps does not depend on any parameter).  Outputs of the iteration:
 *   J   = sum_k w_k S_k            (the expected weighted cost, finite S only)
 *   U'  = sum_k w_k v_k            (Sec. III-D, as oracle_update)
 * Given cotangents gJ (scalar) and gU (T x 2), the vector-Jacobian product
 *   d/dtheta [ gJ J + sum_t gU_t . U'_t ]
 * is returned for theta = the four cost multipliers, the nominal sequence U
 * and the network parameters (packed W1 [H][6], b1 [H], W2 [H][H], b2 [H],
 * W3 [4][H], b3 [4]).  Pieces of the chain:
 *   - Alg. 2: dw_k/dS_j = -(1/lambda) w_k (delta_kj - w_j), so
 *       dJ/dS_j    = w_j (1 - (S_j - J)/lambda),
 *       dU'_t/dS_j = -(w_j/lambda) (v_{j,t} - U'_t);
 *     rho cancels from w (shift invariance) and has no derivative.
 *   - Sec. III-D: U'_t depends on u_t directly through v = u + eps for the
 *     importance samples: dU'_t/du_t = sum_{k importance} w_k.
 *   - Alg. 1 rollout: S_k = sum_{t=1..T} c(x_t, t) + gamma u_{t-1}' Sigma^-1 v_{t-1},
 *     x_t = F(x_{t-1}, g(v_{t-1})) (Sec. V-B), reversed from t = T down to 1.
 *   - Sec. V-C cost: the impulse terms are piecewise constant in x (zero
 *     derivative); the capped track term passes the bilinear slope only when
 *     h <= cap; d zeta/d(v_x, v_y) from zeta = -atan2(v_y, |v_x|) (0 at the
 *     origin).  The clamp g passes the derivative only inside [u_min, u_max].
 * Where S_use is given it replaces the FP64 costs in the weights, J and the
 * cost cotangents (stage-wise checks of a GPU path against its own costs);
 * the trajectories are always the oracle's own.                             */

static double act_deriv(const oracle_problem *P, double h) { return P->activation == 1 ? 1.0 : 1.0 - h * h; }

/* Network part of the step, reversed: given z and dbar = dL/df, accumulate
 * the parameter gradient into gnet and return zbar = dL/dz. */
void oracle_mlp_vjp(const oracle_problem *P, const double z[6], const double dbar[4], double zbar[6],
                    double *gnet) {
  const int H = P->H;
  double h1[ORACLE_MAX_H], h2[ORACLE_MAX_H], h2bar[ORACLE_MAX_H], a2bar[ORACLE_MAX_H], a1bar[ORACLE_MAX_H];
  double *gW1 = gnet, *gb1 = gW1 + 6 * H, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H, *gW3 = gb2 + H,
         *gb3 = gW3 + 4 * H;
  for (int j = 0; j < H; ++j) {
    double a = P->b1[j];
    for (int i = 0; i < 6; ++i) a += P->W1[j * 6 + i] * z[i];
    h1[j] = act(P, a);
  }
  for (int j = 0; j < H; ++j) {
    double a = P->b2[j];
    for (int i = 0; i < H; ++i) a += P->W2[(size_t)j * H + i] * h1[i];
    h2[j] = act(P, a);
  }
  /* output layer d = W3 h2 + b3 */
  for (int o = 0; o < 4; ++o) {
    gb3[o] += dbar[o];
    for (int i = 0; i < H; ++i) gW3[o * H + i] += dbar[o] * h2[i];
  }
  for (int i = 0; i < H; ++i) {
    double s = 0.0;
    for (int o = 0; o < 4; ++o) s += P->W3[o * H + i] * dbar[o];
    h2bar[i] = s;
    a2bar[i] = s * act_deriv(P, h2[i]);
  }
  /* hidden layer 2: a2 = W2 h1 + b2 */
  for (int j = 0; j < H; ++j) {
    gb2[j] += a2bar[j];
    for (int i = 0; i < H; ++i) gW2[(size_t)j * H + i] += a2bar[j] * h1[i];
  }
  for (int i = 0; i < H; ++i) {
    double s = 0.0;
    for (int j = 0; j < H; ++j) s += P->W2[(size_t)j * H + i] * a2bar[j];
    a1bar[i] = s * act_deriv(P, h1[i]);
  }
  /* hidden layer 1: a1 = W1 z + b1 */
  for (int j = 0; j < H; ++j) {
    gb1[j] += a1bar[j];
    for (int m = 0; m < 6; ++m) gW1[j * 6 + m] += a1bar[j] * z[m];
  }
  for (int m = 0; m < 6; ++m) {
    double s = 0.0;
    for (int j = 0; j < H; ++j) s += P->W1[j * 6 + m] * a1bar[j];
    zbar[m] = s;
  }
  (void)h2bar;
}

/* Gradient of the state cost c(x, t) with respect to x (7 entries; only
 * p_x, p_y, v_x, v_y carry one).  comp receives the four unweighted terms as
 * oracle_state_cost does. */
void oracle_state_cost_grad(const oracle_problem *P, const double x[7], int32_t t, double gx[7], double comp[4]) {
  (void)oracle_state_cost(P, x, t, comp, NULL);
  for (int i = 0; i < 7; ++i) gx[i] = 0.0;
  /* track: d h / d(p_x, p_y) of the bilinear lookup, zero where capped */
  double h = oracle_costmap(P, x[0], x[1]);
  if (!(h > P->map_cap)) {
    double fx = (x[0] - P->origin_x) / P->res - 0.5;
    double fy = (x[1] - P->origin_y) / P->res - 0.5;
    double jf = floor(fx), if_ = floor(fy);
    double a = fx - jf, b = fy - if_;
    long W = P->map_w, Hh = P->map_h;
    long j0 = clamp_index(jf, W), j1 = clamp_index(jf + 1.0, W);
    long i0 = clamp_index(if_, Hh), i1 = clamp_index(if_ + 1.0, Hh);
    double m00 = P->map[i0 * W + j0], m01 = P->map[i0 * W + j1];
    double m10 = P->map[i1 * W + j0], m11 = P->map[i1 * W + j1];
    double dh_dfx = (1.0 - b) * (m01 - m00) + b * (m11 - m10);
    double dh_dfy = (1.0 - a) * (m10 - m00) + a * (m11 - m01);
    gx[0] += P->cost_w[0] * dh_dfx / P->res;
    gx[1] += P->cost_w[0] * dh_dfy / P->res;
  }
  /* speed: (v_x - v_des)^2 */
  gx[4] += P->cost_w[1] * 2.0 * (x[4] - P->v_des);
  /* stabilizing: zeta^2, zeta = -atan2(v_y, |v_x|) */
  double vx = x[4], vy = x[5], r2 = vx * vx + vy * vy;
  if (r2 > 0.0) {
    double zeta = -atan2(vy, fabs(vx));
    double sgn = vx > 0.0 ? 1.0 : (vx < 0.0 ? -1.0 : 0.0);
    double dz_dvx = vy * sgn / r2, dz_dvy = -fabs(vx) / r2;
    gx[4] += P->cost_w[2] * 2.0 * zeta * dz_dvx;
    gx[5] += P->cost_w[2] * 2.0 * zeta * dz_dvy;
  }
}

/* One Euler step of Sec. V-B reversed: given x = x_{t-1}, the clamped control
 * gv and xbar_n = dL/dx_t, return xbar = dL/dx_{t-1} (through this step only),
 * gvbar = dL/dg(v), and accumulate the network gradient. */
void oracle_dynamics_step_vjp(const oracle_problem *P, const double x[7], const double gv[2],
                              const double xbar_n[7], double xbar[7], double gvbar[2], double *gnet) {
  const double dt = P->dt, th = x[2], vx = x[4], vy = x[5], c = cos(th), s = sin(th);
  for (int i = 0; i < 7; ++i) xbar[i] = xbar_n[i];
  xbar[2] += dt * (xbar_n[0] * (-s * vx - c * vy) + xbar_n[1] * (c * vx - s * vy));
  xbar[4] += dt * (xbar_n[0] * c + xbar_n[1] * s);
  xbar[5] += dt * (-xbar_n[0] * s + xbar_n[1] * c);
  xbar[6] += dt * xbar_n[2];
  double z[6] = {x[3], x[4], x[5], x[6], gv[0], gv[1]};
  double dbar[4] = {dt * xbar_n[3], dt * xbar_n[4], dt * xbar_n[5], dt * xbar_n[6]};
  double zbar[6];
  oracle_mlp_vjp(P, z, dbar, zbar, gnet);
  for (int i = 0; i < 4; ++i) xbar[3 + i] += zbar[i];
  gvbar[0] = zbar[4];
  gvbar[1] = zbar[5];
}

/* Reverse sweep of one sample (Alg. 1's inner loop backwards) with cost
 * cotangent Sbar: accumulates into gU (T x 2), gnet and gcw (4). */
static void rollout_sample_vjp(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter,
                               int64_t k, double Sbar, double *traj, double *vs, double *gU, double *gnet,
                               double gcw[4]) {
  const int32_t T = P->T;
  int importance = (double)k < (1.0 - P->alpha_explore) * (double)P->K;
  /* forward, keeping x_0..x_T and v_0..v_{T-1} */
  memcpy(traj, x0, 7 * sizeof(double));
  for (int32_t t = 1; t <= T; ++t) {
    double eps[2], gv[2];
    oracle_noise(P, iter, k, t - 1, eps);
    for (int i = 0; i < 2; ++i) {
      vs[2 * (t - 1) + i] = importance ? U[2 * (t - 1) + i] + eps[i] : eps[i];
      gv[i] = clampd(vs[2 * (t - 1) + i], P->u_min[i], P->u_max[i]);
    }
    oracle_dynamics_step(P, traj + 7 * (size_t)(t - 1), gv, traj + 7 * (size_t)t);
  }
  /* backward */
  double xbar[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int32_t t = T; t >= 1; --t) {
    const double *xt = traj + 7 * (size_t)t, *xp = traj + 7 * (size_t)(t - 1), *v = vs + 2 * (t - 1);
    const double *u = U + 2 * (t - 1);
    double gx[7], comp[4];
    oracle_state_cost_grad(P, xt, t, gx, comp);
    for (int i = 0; i < 7; ++i) xbar[i] += Sbar * gx[i];
    for (int i = 0; i < 4; ++i) gcw[i] += Sbar * comp[i];
    double gv[2] = {clampd(v[0], P->u_min[0], P->u_max[0]), clampd(v[1], P->u_min[1], P->u_max[1])};
    double xbar_p[7], gvbar[2];
    oracle_dynamics_step_vjp(P, xp, gv, xbar, xbar_p, gvbar, gnet);
    for (int i = 0; i < 2; ++i) {
      double vbar = (v[i] >= P->u_min[i] && v[i] <= P->u_max[i]) ? gvbar[i] : 0.0;
      double ubar = 0.0;
      if (P->gamma != 0.0) {
        double is2 = 1.0 / (P->sigma[i] * P->sigma[i]);
        /* gamma u_i v_i / sigma_i^2: d/dv = gamma u_i/sigma_i^2, d/du (explicit) = gamma v_i/sigma_i^2 */
        vbar += Sbar * P->gamma * u[i] * is2;
        ubar += Sbar * P->gamma * v[i] * is2;
      }
      if (importance) ubar += vbar;
      gU[2 * (t - 1) + i] += ubar;
    }
    memcpy(xbar, xbar_p, sizeof(xbar));
  }
}

int oracle_net_floats(int32_t H) { return 12 * H + H * H + 4; }

int oracle_iterate_vjp(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter,
                       const double *S_use, double gJ, const double *gUo, double *U_out, double *w, double *S,
                       double *J_out, double *g_cost_w, double *g_U, double *g_net) {
  int rc = check_problem(P);
  if (rc) return rc;
  const int64_t K = P->K;
  const int32_t T = P->T, nf = oracle_net_floats(P->H);
  int nt = P->n_threads > 0 ? P->n_threads : 1;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
  for (int64_t k = 0; k < K; ++k) S[k] = oracle_rollout_sample(P, x0, U, iter, k, NULL, NULL, NULL);
  const double *Sw = S_use ? S_use : S;
  rc = oracle_weights(K, Sw, P->lambda, w, NULL, NULL);
  if (rc) return rc;
  oracle_update(P, iter, w, U, U_out);
  double J = 0.0, w_imp = 0.0, c0 = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    if (w[k] != 0.0) J += w[k] * Sw[k];
    if ((double)k < (1.0 - P->alpha_explore) * (double)K) w_imp += w[k];
  }
  *J_out = J;
  if (gUo)
    for (int32_t t = 0; t < 2 * T; ++t) c0 += gUo[t] * U_out[t];
  for (int i = 0; i < 4; ++i) g_cost_w[i] = 0.0;
  for (int32_t t = 0; t < 2 * T; ++t) g_U[t] = gUo ? gUo[t] * w_imp : 0.0;
  for (int32_t i = 0; i < nf; ++i) g_net[i] = 0.0;
  /* per-thread accumulators, summed in thread order afterwards */
  double *acc = (double *)calloc((size_t)nt * (nf + 2 * T + 4), sizeof(double));
  double *work = (double *)malloc((size_t)nt * (7 * (T + 1) + 2 * T) * sizeof(double));
  if (!acc || !work) {
    free(acc);
    free(work);
    return ORACLE_ERR_ARG;
  }
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int id = omp_get_thread_num();
#else
    int id = 0;
#endif
    double *gnet = acc + (size_t)id * (nf + 2 * T + 4), *gU = gnet + nf, *gcw = gU + 2 * T;
    double *traj = work + (size_t)id * (7 * (T + 1) + 2 * T), *vs = traj + 7 * (T + 1);
#pragma omp for schedule(dynamic, 4)
    for (int64_t k = 0; k < K; ++k) {
      if (w[k] == 0.0) continue;
      int importance = (double)k < (1.0 - P->alpha_explore) * (double)K;
      double a = 0.0; /* sum_t gU_t . v_{k,t} */
      if (gUo) {
        for (int32_t t = 0; t < T; ++t) {
          double eps[2];
          oracle_noise(P, iter, k, t, eps);
          for (int i = 0; i < 2; ++i) a += gUo[2 * t + i] * (importance ? U[2 * t + i] + eps[i] : eps[i]);
        }
      }
      double Sbar = w[k] * (gJ * (1.0 - (Sw[k] - J) / P->lambda) - (a - c0) / P->lambda);
      rollout_sample_vjp(P, x0, U, iter, k, Sbar, traj, vs, gU, gnet, gcw);
    }
  }
  for (int id = 0; id < nt; ++id) {
    const double *gnet = acc + (size_t)id * (nf + 2 * T + 4), *gU = gnet + nf, *gcw = gU + 2 * T;
    for (int32_t i = 0; i < nf; ++i) g_net[i] += gnet[i];
    for (int32_t t = 0; t < 2 * T; ++t) g_U[t] += gU[t];
    for (int i = 0; i < 4; ++i) g_cost_w[i] += gcw[i];
  }
  free(acc);
  free(work);
  return ORACLE_OK;
}

/* ========================================================================= */
/* Closed loop (the end of Alg. 1's outer loop).
 *
 * Control smoothing (Sec. III-E, "Control Smoothing"): fit, at every step j,
 * a polynomial of degree `deg` to the 2 half + 1 values around j by least
 * squares and keep its value at j -- the Savitzky-Golay filter (Savitzky &
 * Golay, Anal. Chem. 36, 1964).  The paper does not give the window or the
 * degree; half = 2 and deg = 2 are taken.  Edge steps replicate the first /
 * last value of the sequence to fill the window.  The fit is computed here
 * from its definition (normal equations of the local least-squares problem,
 * solved by Gaussian elimination) for each window.                           */
static int solve_small(int n, double *A, double *b) {
  /* Gaussian elimination with partial pivoting on the n x n row-major A */
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return -1;
    if (p != c) {
      for (int k = 0; k < n; ++k) {
        double t = A[c * n + k];
        A[c * n + k] = A[p * n + k];
        A[p * n + k] = t;
      }
      double t = b[c];
      b[c] = b[p];
      b[p] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return 0;
}

/* y[j] = value at j of the least-squares polynomial of degree deg through
 * x[j - half .. j + half] (indices clamped to [0, n-1]), one channel of a
 * sequence with stride `stride`. */
int oracle_savgol(int32_t n, int32_t stride, const double *x, int32_t half, int32_t deg, double *y) {
  if (n < 1 || half < 0 || deg < 0 || deg > 2 * half || deg > 8) return ORACLE_ERR_ARG;
  const int m = deg + 1;
  for (int32_t j = 0; j < n; ++j) {
    double A[81], b[9];
    for (int r = 0; r < m; ++r) {
      b[r] = 0.0;
      for (int c = 0; c < m; ++c) A[r * m + c] = 0.0;
    }
    for (int32_t o = -half; o <= half; ++o) {
      int32_t i = j + o;
      i = i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
      double pw[9];
      pw[0] = 1.0;
      for (int r = 1; r < m; ++r) pw[r] = pw[r - 1] * (double)o;  /* basis 1, o, o^2 ... */
      for (int r = 0; r < m; ++r) {
        b[r] += pw[r] * x[(size_t)i * stride];
        for (int c = 0; c < m; ++c) A[r * m + c] += pw[r] * pw[c];
      }
    }
    if (solve_small(m, A, b)) return ORACLE_ERR_ARG;
    y[(size_t)j * stride] = b[0]; /* the polynomial's value at offset 0 */
  }
  return ORACLE_OK;
}

/* One closed-loop step: the iteration, then (Alg. 1, after ComputeWeights)
 *   smoothing 0: U_s = U'                         (no filter)
 *   smoothing 1: U_s = SGF(U')                    (Sec. III-E: filter the weighted mean)
 *   smoothing 2: U_s = U + SGF(U' - U)            (Alg. 1: U <- U + SGF * sum_k w_k eps_k,
 *                                                  the same when alpha = 0)
 *   u_applied   = U_s[0]                          ("SendToActuators")
 *   x_next      = F(x0, g(u_applied)) if plant    (noise-free model as the plant)
 *   U_next[t-1] = U_s[t], U_next[T-1] = (0, 0)    (warm start; Initialize = (0, 0)
 *                                                  in the paper's parameter table)
 * S_use (optional, K) replaces the costs in the weights (stage-wise checks).  */
int oracle_control_step(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter,
                        const double *S_use, int32_t smoothing, int32_t plant, double *x_next, double *U_next,
                        double u_applied[2], double *U_prime) {
  int rc = check_problem(P);
  if (rc) return rc;
  const int32_t T = P->T;
  double *w = (double *)malloc(sizeof(double) * (size_t)P->K);
  double *S = (double *)malloc(sizeof(double) * (size_t)P->K);
  double *Us = (double *)malloc(sizeof(double) * 2 * (size_t)T);
  double *D = (double *)malloc(sizeof(double) * 2 * (size_t)T);
  if (!w || !S || !Us || !D) {
    free(w); free(S); free(Us); free(D);
    return ORACLE_ERR_ARG;
  }
  int nt = P->n_threads > 0 ? P->n_threads : 1;
  (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
  for (int64_t k = 0; k < P->K; ++k) S[k] = oracle_rollout_sample(P, x0, U, iter, k, NULL, NULL, NULL);
  rc = oracle_weights(P->K, S_use ? S_use : S, P->lambda, w, NULL, NULL);
  if (rc == ORACLE_OK) {
    oracle_update(P, iter, w, U, U_prime);
    if (smoothing == 1) {
      for (int i = 0; i < 2 && rc == ORACLE_OK; ++i) rc = oracle_savgol(T, 2, U_prime + i, 2, 2, Us + i);
    } else if (smoothing == 2) {
      for (int32_t t = 0; t < 2 * T; ++t) D[t] = U_prime[t] - U[t];
      for (int i = 0; i < 2 && rc == ORACLE_OK; ++i) rc = oracle_savgol(T, 2, D + i, 2, 2, Us + i);
      for (int32_t t = 0; t < 2 * T; ++t) Us[t] += U[t];
    } else {
      memcpy(Us, U_prime, sizeof(double) * 2 * (size_t)T);
    }
  }
  if (rc == ORACLE_OK) {
    u_applied[0] = Us[0];
    u_applied[1] = Us[1];
    if (plant) oracle_plant_step(P, x0, u_applied, x_next);
    else memcpy(x_next, x0, 7 * sizeof(double));
    for (int32_t t = 1; t < T; ++t) {
      U_next[2 * (t - 1)] = Us[2 * t];
      U_next[2 * (t - 1) + 1] = Us[2 * t + 1];
    }
    U_next[2 * (T - 1)] = 0.0;
    U_next[2 * (T - 1) + 1] = 0.0;
  }
  free(w); free(S); free(Us); free(D);
  return rc;
}

/* ========================================================================= */
/* Cross-entropy weights (Alg. 3, "Compute Weights (Cross Entropy)"), the
 * paper's comparison controller on the same rollouts:
 *   zeta = round(K (1 - delta)),  Z = the zeta-th smallest cost,
 *   w_k  = 1/|E| for k in the elite set E = {k : S_k <= Z}, else 0.
 * Readings: the printed indicator I{S_k < Z} would keep zeta - 1 samples and
 * weights summing to (zeta - 1)/zeta; the elite set of the method's own
 * definition ({C <= gamma}, Sec. VI-A, step 3) is taken, normalised by its size
 * (= zeta without ties) so that the weights sum to one.  round() is
 * floor(x + 1/2); zeta is clamped to [1, number of finite costs]; non-finite
 * costs are never elite.  The ranks come from a plain insertion sort of the
 * finite costs.                                                              */
int oracle_cem_weights(int64_t K, const double *S, double delta, double *w, double *Z_out, int64_t *n_elite) {
  if (K <= 0 || !(delta >= 0.0 && delta <= 1.0)) return ORACLE_ERR_ARG;
  double *f = (double *)malloc(sizeof(double) * (size_t)K);
  if (!f) return ORACLE_ERR_ARG;
  int64_t n = 0;
  for (int64_t k = 0; k < K; ++k) {
    if (!isfinite(S[k])) continue;
    int64_t i = n++;
    while (i > 0 && f[i - 1] > S[k]) {
      f[i] = f[i - 1];
      --i;
    }
    f[i] = S[k];
  }
  if (n == 0) {
    free(f);
    for (int64_t k = 0; k < K; ++k) w[k] = 0.0;
    return ORACLE_ERR_NONFINITE;
  }
  int64_t zeta = (int64_t)floor((double)K * (1.0 - delta) + 0.5);
  if (zeta < 1) zeta = 1;
  if (zeta > n) zeta = n;
  const double Z = f[zeta - 1];
  free(f);
  int64_t m = 0;
  for (int64_t k = 0; k < K; ++k) m += (isfinite(S[k]) && S[k] <= Z) ? 1 : 0;
  for (int64_t k = 0; k < K; ++k) w[k] = (isfinite(S[k]) && S[k] <= Z) ? 1.0 / (double)m : 0.0;
  if (Z_out) *Z_out = Z;
  if (n_elite) *n_elite = m;
  return ORACLE_OK;
}

/* One cross-entropy MPC iteration: the rollouts of Alg. 1, the weights of
 * Alg. 3 and the same control law (U' = sum_k w_k v_k, the un-weighted mean of
 * the elite controls).  S_use replaces the costs in the weights (stage-wise). */
int oracle_iterate_cem(const oracle_problem *P, const double x0[7], const double *U, uint64_t iter, double delta,
                       const double *S_use, double *U_out, double *w, double *S) {
  int rc = check_problem(P);
  if (rc) return rc;
  int nt = P->n_threads > 0 ? P->n_threads : 1;
  (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
  for (int64_t k = 0; k < P->K; ++k) S[k] = oracle_rollout_sample(P, x0, U, iter, k, NULL, NULL, NULL);
  rc = oracle_cem_weights(P->K, S_use ? S_use : S, delta, w, NULL, NULL);
  if (rc) return rc;
  oracle_update(P, iter, w, U, U_out);
  return ORACLE_OK;
}
