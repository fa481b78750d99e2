"""Mutation check of the oracle's pins.

Each entry below plants one plausible mistake in a copy of ``oracle/itmpc_oracle.c``:
a dropped term, a flipped sign, a wrong, swapped or transposed index, an off-by-one,
a wrong constant.  The copy is compiled like the oracle and the pin tests that cover
that part of the oracle run against it (``ITMPC_ORACLE_LIB``) in a subprocess.  Every
mutant must make at least one of those pins fail; the unmutated source, compiled and
run the same way, must pass them.  The oracle's own source is never modified.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NOISE = ["tests/test_oracle_noise.py"]
DYN = ["tests/test_oracle_dynamics.py"]
COST = ["tests/test_oracle_costs.py"]
WU = ["tests/test_oracle_weights_update.py"]
LOOP = ["tests/test_oracle_closed_loop.py"]
CEM = ["tests/test_oracle_cem.py"]
BASIS = ["tests/test_oracle_basis.py"]
ADJ = ["tests/test_oracle_adjoint.py"]

# (name, text in the oracle, replacement, pin files, occurrences of the text, which one to replace)
MUTANTS = [
    # Philox-4x32-10, Box-Muller, the noise counter (Sec. II sampling; Salmon et al.; Box & Muller)
    ("philox_weyl_constant", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;", NOISE),
    ("philox_lane_swap", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;", NOISE),
    ("philox_nine_rounds", "round < 10; ++round", "round < 9; ++round", NOISE),
    ("uniform_offset", "((double)(a >> 8) + 1.0)", "((double)(a >> 8) + 0.5)", NOISE),
    ("box_muller_cos_sin", "z[0] = r * cos(two_pi * u1);", "z[0] = r * sin(two_pi * u1);", NOISE),
    ("box_muller_radius", "sqrt(-2.0 * log(u0))", "sqrt(-log(u0))", NOISE),
    ("sigma_index", "eps[1] = P->sigma[1] * z[1];", "eps[1] = P->sigma[0] * z[1];", NOISE),
    ("counter_k_t_swapped", "{(uint32_t)k, (uint32_t)t,", "{(uint32_t)t, (uint32_t)k,", NOISE),
    ("counter_instance_shift", "| (P->instance << 16)}", "| (P->instance << 8)}", NOISE),
    # network and equations of motion (Sec. V-B)
    ("mlp_w2_transposed",
     "a += P->W2[(size_t)j * H + i] * h1[i];\n    h2[j] = act(P, a);\n  }\n  for (int o = 0; o < 4; ++o) {",
     "a += P->W2[(size_t)i * H + j] * h1[i];\n    h2[j] = act(P, a);\n  }\n  for (int o = 0; o < 4; ++o) {", DYN),
    ("mlp_b2_dropped", "double a = P->b2[j];", "double a = 0.0;", DYN, 2, 0),
    ("mlp_w1_input_reversed", "a += P->W1[j * 6 + i] * z[i];", "a += P->W1[j * 6 + i] * z[5 - i];", DYN, 2, 0),
    ("mlp_output_no_bias", "double a = P->b3[o];", "double a = 0.0;", DYN),
    ("kinematics_px_sign", "(cos(th) * vx - sin(th) * vy) * P->dt", "(cos(th) * vx + sin(th) * vy) * P->dt", DYN),
    ("kinematics_py_sin_cos", "(sin(th) * vx + cos(th) * vy) * P->dt", "(cos(th) * vx + sin(th) * vy) * P->dt", DYN),
    ("yaw_without_dt", "xn[2] = x[2] + thd * P->dt;", "xn[2] = x[2] + thd;", DYN),
    ("network_input_order", "double z[6] = {x[3], x[4], x[5], x[6], gv[0], gv[1]};",
     "double z[6] = {x[4], x[3], x[5], x[6], gv[0], gv[1]};", DYN, 2, 0),
    ("network_control_order", "double z[6] = {x[3], x[4], x[5], x[6], gv[0], gv[1]};",
     "double z[6] = {x[3], x[4], x[5], x[6], gv[1], gv[0]};", DYN, 2, 0),
    # costmap and state cost (Sec. V-C)
    ("texel_centre", "double fx = (px - P->origin_x) / P->res - 0.5;", "double fx = (px - P->origin_x) / P->res;",
     COST),
    ("bilinear_weight", "+ a * (1.0 - b) * m01 +", "+ b * (1.0 - a) * m01 +", COST),
    ("map_rows_cols", "double m00 = P->map[i0 * W + j0], m01 = P->map[i0 * W + j1];",
     "double m00 = P->map[i0 * W + j0], m01 = P->map[i1 * W + j0];", COST, 2, 0),
    ("y_uses_origin_x", "double fy = (py - P->origin_y) / P->res - 0.5;",
     "double fy = (py - P->origin_x) / P->res - 0.5;", COST),
    ("map_cap_dropped", "if (h > P->map_cap) h = P->map_cap;", "", COST),
    ("speed_not_squared", "double speed = (vx - P->v_des) * (vx - P->v_des);", "double speed = (vx - P->v_des);", COST),
    ("track_threshold_not_strict", "if (h > P->track_thresh) imp", "if (h >= P->track_thresh) imp", COST),
    ("impulse_decay_off_by_one", "imp += pow(P->crash_decay, (double)t) * P->crash_cost;",
     "imp += pow(P->crash_decay, (double)(t - 1)) * P->crash_cost;", COST),
    ("slip_without_abs_vx", "double zeta = -atan2(vy, fabs(vx));\n  double speed",
     "double zeta = -atan2(vy, vx);\n  double speed", COST),
    ("slip_threshold_signed", "if (fabs(zeta) > P->slip_thresh) imp", "if (zeta > P->slip_thresh) imp", COST),
    ("cost_weights_swapped", "P->cost_w[1] * speed + P->cost_w[2] * zeta * zeta",
     "P->cost_w[2] * speed + P->cost_w[1] * zeta * zeta", COST),
    ("cost_time_index", "double c = oracle_state_cost(P, x, t, c4, &m);",
     "double c = oracle_state_cost(P, x, t - 1, c4, &m);", COST),
    # Alg. 1 rollout, Alg. 2 weights, the update of Sec. III-D, the control cost of Sec. III-E
    ("rollout_noise_index", "oracle_noise(P, iter, k, t - 1, eps);", "oracle_noise(P, iter, k, t, eps);", WU, 2, 0),
    ("weights_not_normalised", "exp(-(S[k] - rho) / lambda) / eta : 0.0;", "exp(-(S[k] - rho) / lambda) : 0.0;", WU),
    ("weights_sign", "exp(-(S[k] - rho) / lambda) / eta : 0.0;", "exp((S[k] - rho) / lambda) / eta : 0.0;", WU),
    ("weights_lambda_dropped", "w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) / eta",
     "w[k] = isfinite(S[k]) ? exp(-(S[k] - rho)) / eta", WU),
    ("update_exploration_split", "int importance = (double)k < (1.0 - P->alpha_explore) * (double)P->K;\n      double v0",
     "int importance = (double)k <= (1.0 - P->alpha_explore) * (double)P->K;\n      double v0", WU),
    ("rollout_exploration_split", "int importance = (double)k < (1.0 - P->alpha_explore) * (double)P->K;\n  double S",
     "int importance = (double)k <= (1.0 - P->alpha_explore) * (double)P->K;\n  double S", WU),
    ("update_channel", "s1 += w[k] * v1;", "s1 += w[k] * v0;", WU),
    ("update_exploration_adds_U", "double v1 = importance ? U[2 * t + 1] + eps[1] : eps[1];",
     "double v1 = U[2 * t + 1] + eps[1];", WU),
    ("control_cost_sigma", "U[2 * (t - 1)] * v[0] / (P->sigma[0] * P->sigma[0])", "U[2 * (t - 1)] * v[0] / P->sigma[0]",
     WU),
    ("control_cost_dropped", "S += c + P->gamma * ctrl;", "S += c;", WU),
    # Savitzky-Golay smoothing and the closed-loop step (Sec. III-E, Alg. 1)
    ("savgol_basis_shift", "pw[r] = pw[r - 1] * (double)o;", "pw[r] = pw[r - 1] * (double)(o + 1);", LOOP),
    ("savgol_mirror_edges", "i = i < 0 ? 0 : (i > n - 1 ? n - 1 : i);",
     "i = i < 0 ? -i : (i > n - 1 ? 2 * (n - 1) - i : i);", LOOP),
    ("warm_start_keeps_last", "U_next[2 * (T - 1)] = 0.0;", "U_next[2 * (T - 1)] = Us[2 * (T - 1)];", LOOP),
    ("applied_control_unsmoothed", "u_applied[0] = Us[0];", "u_applied[0] = U_prime[0];", LOOP),
    ("delta_smoothing_without_U", "for (int32_t t = 0; t < 2 * T; ++t) Us[t] += U[t];", "", LOOP),
    # cross-entropy weights (Alg. 3)
    ("cem_strict_elite", "w[k] = (isfinite(S[k]) && S[k] <= Z)", "w[k] = (isfinite(S[k]) && S[k] < Z)", CEM),
    ("cem_floor_not_round", "floor((double)K * (1.0 - delta) + 0.5)", "floor((double)K * (1.0 - delta))", CEM),
    ("cem_delta_direction", "floor((double)K * (1.0 - delta) + 0.5)", "floor((double)K * delta + 0.5)", CEM),
    # basis-function model (Sec. V-B, appendix)
    ("basis_phi5_vx", "phi[5] = r * vy / 25.0;", "phi[5] = r * vx / 25.0;", BASIS),
    ("basis_front_slip_sign", "atan(vy / vx + 0.45 * r / vx - ud)", "atan(vy / vx - 0.45 * r / vx - ud)", BASIS),
    ("basis_low_speed_sign", ": -ud;", ": ud;", BASIS),
    ("basis_theta_transposed", "a += P->theta[i * 4 + o] * phi[i];", "a += P->theta[o * 25 + i] * phi[i];", BASIS),
    ("basis_phi21_scale", "phi[21] = vx * vx / 100.0;", "phi[21] = vx * vx / 10.0;", BASIS),
    # the adjoint (reverse mode of the above)
    ("adj_tanh_derivative", "1.0 - h * h;", "1.0 - h;", ADJ),
    ("adj_w2_backprop_transposed", "s += P->W2[(size_t)j * H + i] * a2bar[j];",
     "s += P->W2[(size_t)i * H + j] * a2bar[j];", ADJ),
    ("adj_speed_gradient_factor", "gx[4] += P->cost_w[1] * 2.0 * (x[4] - P->v_des);",
     "gx[4] += P->cost_w[1] * (x[4] - P->v_des);", ADJ),
    ("adj_map_slope_y_weights", "double dh_dfy = (1.0 - a) * (m10 - m00) + a * (m11 - m01);",
     "double dh_dfy = (1.0 - b) * (m10 - m00) + b * (m11 - m01);", ADJ),
    ("adj_cost_cotangent_J_sign", "gJ * (1.0 - (Sw[k] - J) / P->lambda)", "gJ * (1.0 + (Sw[k] - J) / P->lambda)", ADJ),
    ("adj_cost_cotangent_U_sign", "- (a - c0) / P->lambda);", "+ (a - c0) / P->lambda);", ADJ),
    ("adj_clamp_passes_gradient", "(v[i] >= P->u_min[i] && v[i] <= P->u_max[i]) ? gvbar[i] : 0.0", "gvbar[i]", ADJ),
    ("adj_exploration_gets_dU", "if (importance) ubar += vbar;", "ubar += vbar;", ADJ),
    ("adj_direct_dU_without_w_imp", "g_U[t] = gUo ? gUo[t] * w_imp : 0.0;", "g_U[t] = gUo ? gUo[t] : 0.0;", ADJ),
    ("adj_heading_sign", "xbar_n[0] * (-s * vx - c * vy)", "xbar_n[0] * (s * vx - c * vy)", ADJ),
    ("adj_yaw_rate_dropped", "xbar[6] += dt * xbar_n[2];", "", ADJ),
    ("adj_cost_weight_grad_unscaled", "gcw[i] += Sbar * comp[i];", "gcw[i] += comp[i];", ADJ),
    ("adj_control_cost_du_dropped", "ubar += Sbar * P->gamma * v[i] * is2;", "", ADJ),
    ("adj_slip_slope_sign", "dz_dvy = -fabs(vx) / r2;", "dz_dvy = fabs(vx) / r2;", ADJ),
    ("adj_gW2_transposed", "gW2[(size_t)j * H + i] += a2bar[j] * h1[i];", "gW2[(size_t)i * H + j] += a2bar[j] * h1[i];",
     ADJ),
    ("adj_gb1_dropped", "gb1[j] += a1bar[j];", "", ADJ),
    # the sort of the cross-entropy ranks and the Savitzky-Golay solve
    ("cem_sort_descending", "while (i > 0 && f[i - 1] > S[k])", "while (i > 0 && f[i - 1] < S[k])", CEM),
    ("savgol_back_substitution", "b[c] = s / A[c * n + c];", "b[c] = s;", LOOP),
    ("rollout_clamp_dropped", "gv[i] = clampd(v[i], P->u_min[i], P->u_max[i]);", "gv[i] = v[i];", WU),
    ("weights_eta_counts_nonfinite", "eta += isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 0.0;",
     "eta += isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 1.0;", WU),
    ("weights_rho_first_finite", "if (isfinite(S[k]) && S[k] < rho) rho = S[k];",
     "if (isfinite(S[k]) && rho == INFINITY) rho = S[k];", WU),
    ("update_noise_next_step", "      oracle_noise(P, iter, k, t, eps);\n      int importance",
     "      oracle_noise(P, iter, k, t + 1 < P->T ? t + 1 : t, eps);\n      int importance", WU),
    ("rollout_margin_not_tracked", "if (m < mmin) mmin = m;", "", COST),
    ("rollout_margin_last_step", "if (m < mmin) mmin = m;", "mmin = m;", COST),
    ("mlp_h1_no_tanh", "    h1[j] = act(P, a);", "    h1[j] = a;", DYN, 2, 0),
    ("mlp_h2_no_tanh", "    h2[j] = act(P, a);", "    h2[j] = a;", DYN, 2, 0),
    ("mlp_w3_reads_h1", "a += P->W3[(size_t)o * H + i] * h2[i];", "a += P->W3[(size_t)o * H + i] * h1[i];", DYN),
    ("position_uses_new_heading", "xn[1] = x[1] + (sin(th) * vx + cos(th) * vy) * P->dt;",
     "xn[1] = x[1] + (sin(th + thd * P->dt) * vx + cos(th + thd * P->dt) * vy) * P->dt;", DYN),
    ("state_derivative_without_dt", "xn[3 + i] = x[3 + i] + f[i] * P->dt;", "xn[3 + i] = x[3 + i] + f[i];", DYN),
    ("plant_without_clamp",
     "double gv[2] = {clampd(u[0], P->u_min[0], P->u_max[0]), clampd(u[1], P->u_min[1], P->u_max[1])};",
     "double gv[2] = {u[0], u[1]};", DYN + LOOP),
    ("clamp_bounds_swapped", "return v < lo ? lo : (v > hi ? hi : v);", "return v < lo ? hi : (v > hi ? lo : v);",
     DYN + WU),
    ("costmap_clamp_high_edge", "(i > (double)(n - 1) ? n - 1 : (long)i)", "(i > (double)(n - 1) ? n - 2 : (long)i)",
     COST),
    ("costmap_floor_truncates", "double jf = floor(fx), if_ = floor(fy);",
     "double jf = (double)(long)fx, if_ = (double)(long)fy;", COST, 2, 0),
    ("box_muller_z1_cos", "z[1] = r * sin(two_pi * u1);", "z[1] = r * cos(two_pi * u1);", NOISE),
    ("noise_seed_halves_swapped", "uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)(P->seed >> 32), (uint32_t)P->seed};", NOISE),
    ("noise_iter_hi_mask", "(uint32_t)((iter >> 32) & 0xFFFFu)", "(uint32_t)((iter >> 32) & 0xFFu)", NOISE),
    ("noise_iter_lo_dropped", "{(uint32_t)k, (uint32_t)t, (uint32_t)iter,", "{(uint32_t)k, (uint32_t)t, 0u,", NOISE),
    ("basis_alpha_r_sign", "atan(vy / vx - 0.35 * r / vx)", "atan(vy / vx + 0.35 * r / vx)", BASIS),
    ("basis_slow_threshold", "const int fast = vx > 0.1;", "const int fast = vx > 0.0;", BASIS),
    ("basis_phi24_square", "phi[24] = uF * uF * uF;", "phi[24] = uF * uF;", BASIS),
    ("basis_phi3_abs_dropped", "phi[3] = sd * tf * fabs(tf) / (1200.0 * 1200.0);",
     "phi[3] = sd * tf * tf / (1200.0 * 1200.0);", BASIS),
    ("adj_h1_no_tanh", "    h1[j] = act(P, a);", "    h1[j] = a;", ADJ, 2, 1),
    ("adj_h2_no_tanh", "    h2[j] = act(P, a);", "    h2[j] = a;", ADJ, 2, 1),
    ("adj_costmap_floor_truncates", "double jf = floor(fx), if_ = floor(fy);",
     "double jf = (double)(long)fx, if_ = (double)(long)fy;", ADJ, 2, 1),
    ("savgol_value_is_slope", "y[(size_t)j * stride] = b[0];", "y[(size_t)j * stride] = b[1];", LOOP),
    ("savgol_stride_ignored", "b[r] += pw[r] * x[(size_t)i * stride];", "b[r] += pw[r] * x[(size_t)i];", LOOP),
    ("savgol_window_short", "for (int32_t o = -half; o <= half; ++o) {", "for (int32_t o = -half; o < half; ++o) {",
     LOOP),
    ("delta_smoothing_without_difference", "      for (int32_t t = 0; t < 2 * T; ++t) D[t] = U_prime[t] - U[t];",
     "      for (int32_t t = 0; t < 2 * T; ++t) D[t] = U_prime[t];", LOOP),
    ("applied_throttle_from_next_step", "    u_applied[1] = Us[1];", "    u_applied[1] = Us[3];", LOOP),
    ("warm_start_shift_by_two", "      U_next[2 * (t - 1)] = Us[2 * t];\n",
     "      U_next[2 * (t - 1)] = Us[2 * t < 2 * T - 2 ? 2 * t + 2 : 2 * t];\n", LOOP),
    ("plant_driven_by_next_control", "    if (plant) oracle_plant_step(P, x0, u_applied, x_next);",
     "    if (plant) oracle_plant_step(P, x0, Us + 2, x_next);", LOOP),
    ("cem_zeta_not_clamped_low", "  if (zeta < 1) zeta = 1;\n", "", CEM),
    ("cem_zeta_clamped_to_K", "  if (zeta > n) zeta = n;\n", "  if (zeta > K) zeta = K;\n", CEM),
    ("cem_minus_inf_counted", "m += (isfinite(S[k]) && S[k] <= Z) ? 1 : 0;", "m += (S[k] <= Z) ? 1 : 0;", CEM),
    ("cem_weight_not_normalised", "? 1.0 / (double)m : 0.0;", "? 1.0 : 0.0;", CEM),
    ("cem_given_costs_ignored", "rc = oracle_cem_weights(P->K, S_use ? S_use : S, delta, w, NULL, NULL);",
     "rc = oracle_cem_weights(P->K, S, delta, w, NULL, NULL);", CEM),
    ("adj_gb3_dropped", "    gb3[o] += dbar[o];\n",
     "", ADJ),
    ("adj_gW3_uses_h1", "for (int i = 0; i < H; ++i) gW3[o * H + i] += dbar[o] * h2[i];",
     "for (int i = 0; i < H; ++i) gW3[o * H + i] += dbar[o] * h1[i];", ADJ),
    ("adj_h2_derivative_uses_h1", "a2bar[i] = s * act_deriv(P, h2[i]);",
     "a2bar[i] = s * act_deriv(P, h1[i]);", ADJ),
    ("adj_gb2_dropped", "    gb2[j] += a2bar[j];\n",
     "", ADJ),
    ("adj_gW1_input_index", "for (int m = 0; m < 6; ++m) gW1[j * 6 + m] += a1bar[j] * z[m];",
     "for (int m = 0; m < 6; ++m) gW1[j * 6 + m] += a1bar[j] * z[5 - m];", ADJ),
    ("adj_zbar_transposed", "for (int j = 0; j < H; ++j) s += P->W1[j * 6 + m] * a1bar[j];",
     "for (int j = 0; j < H; ++j) s += P->W1[(j * 6 + m) % (6 * H)] * a1bar[(j + 1) % H];", ADJ),
    ("adj_map_slope_no_res", "gx[0] += P->cost_w[0] * dh_dfx / P->res;",
     "gx[0] += P->cost_w[0] * dh_dfx;", ADJ),
    ("adj_map_slope_through_cap", "  if (!(h > P->map_cap)) {\n    double fx",
     "  if (1) {\n    double fx", ADJ),
    ("adj_slip_dvx_sign", "double dz_dvx = vy * sgn / r2,",
     "double dz_dvx = -vy * sgn / r2,", ADJ),
    ("adj_vx_through_heading", "xbar[4] += dt * (xbar_n[0] * c + xbar_n[1] * s);",
     "xbar[4] += dt * (xbar_n[0] * c - xbar_n[1] * s);", ADJ),
    ("adj_vy_through_heading", "xbar[5] += dt * (-xbar_n[0] * s + xbar_n[1] * c);",
     "xbar[5] += dt * (xbar_n[0] * s + xbar_n[1] * c);", ADJ),
    ("adj_dbar_without_dt", "double dbar[4] = {dt * xbar_n[3], dt * xbar_n[4], dt * xbar_n[5], dt * xbar_n[6]};",
     "double dbar[4] = {xbar_n[3], xbar_n[4], xbar_n[5], xbar_n[6]};", ADJ),
    ("adj_state_skips_network", "  for (int i = 0; i < 4; ++i) xbar[3 + i] += zbar[i];\n",
     "", ADJ),
    ("adj_controls_swapped", "  gvbar[0] = zbar[4];\n  gvbar[1] = zbar[5];",
     "  gvbar[0] = zbar[5];\n  gvbar[1] = zbar[4];", ADJ),
    ("adj_cost_at_previous_state", "    oracle_state_cost_grad(P, xt, t, gx, comp);",
     "    oracle_state_cost_grad(P, xp, t, gx, comp);", ADJ),
    ("adj_control_cost_du_uses_u", "        ubar += Sbar * P->gamma * v[i] * is2;",
     "        ubar += Sbar * P->gamma * u[i] * is2;", ADJ),
    ("adj_J_includes_zero_weights", "    if (w[k] != 0.0) J += w[k] * Sw[k];",
     "    J += w[k] * Sw[k];", ADJ),
    ("adj_c0_dropped", "    for (int32_t t = 0; t < 2 * T; ++t) c0 += gUo[t] * U_out[t];",
     "    for (int32_t t = 0; t < 2 * T; ++t) c0 += 0.0;", ADJ),
    ("philox_k0_weyl_constant", "k0 += 0x9E3779B9u;",
     "k0 += 0x9E3779B8u;", NOISE),
    ("philox_multiplier0", "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
     "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;", NOISE),
    ("philox_lo_words_swapped", "    uint32_t n1 = lo1;\n",
     "    uint32_t n1 = lo0;\n", NOISE),
    ("philox_key_bump_first_round", "    if (round > 0) {\n",
     "    if (round >= 0) {\n", NOISE),
    ("uniform_bits_shift", "static double u01(uint32_t a) { return ((double)(a >> 8) + 1.0) * (1.0 / 16777216.0); }",
     "static double u01(uint32_t a) { return ((double)(a >> 9) + 1.0) * (1.0 / 8388608.0); }", NOISE),
    ("box_muller_two_pi_as_pi", "  z[0] = r * cos(two_pi * u1);",
     "  z[0] = r * cos(0.5 * two_pi * u1);", NOISE),
    ("noise_words_2_3", "  oracle_box_muller(w[0], w[1], z);",
     "  oracle_box_muller(w[2], w[3], z);", NOISE),
    ("dyn_heading_uses_yaw_of_xd", "  double th = x[2], vx = x[4], vy = x[5], thd = x[6];\n  double z[6]",
     "  double th = x[2], vx = x[4], vy = x[5], thd = x[3];\n  double z[6]", DYN),
    ("basis_theta_row_stride", "a += P->theta[i * 4 + o] * phi[i];",
     "a += P->theta[i * 4 + (o + 1) % 4] * phi[i];", BASIS),
    ("basis_phi19_scale", "phi[19] = th * vx / 3.0;",
     "phi[19] = th * vx / 30.0;", BASIS),
    ("basis_phi9_slow_branch", "phi[9] = fast ? (vy / vx) / 40.0 : 0.0;",
     "phi[9] = (vy / (vx == 0.0 ? 1.0 : vx)) / 40.0;", BASIS),
]


def _mutate(src, old, new, count=1, nth=0):
    assert src.count(old) == count, f"expected {count} occurrence(s) of {old!r} in the oracle"
    i = -1
    for _ in range(nth + 1):
        i = src.index(old, i + 1)
    return src[:i] + new + src[i + len(old):]


def _build_and_run(text, lib, files):
    """Compile `text` like the oracle into `lib`, run the pin files against it; pytest's return code."""
    c_file = lib[:-3] + ".c"
    with open(c_file, "w") as f:
        f.write(text)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", lib, c_file, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, ITMPC_ORACLE_LIB=lib, OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *files], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(oracle.SOURCE).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    texts = {m[0]: _mutate(src, *m[1:3], *m[4:]) for m in MUTANTS}  # fails here if the oracle text moved
    files_all = sorted({f for m in MUTANTS for f in m[3]})
    workers = max(1, min(8, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        control = ex.submit(_build_and_run, src, str(tmp_path / "control.so"), files_all)
        runs = {m[0]: ex.submit(_build_and_run, texts[m[0]], str(tmp_path / f"{m[0]}.so"), m[3]) for m in MUTANTS}
        assert control.result() == 0, "the unmutated oracle must pass its pins under the same harness"
        codes = {n: f.result() for n, f in runs.items()}
    # 1: a pin failed; negative: the mutant crashed the test process (also a detection)
    survivors = {n: rc for n, rc in codes.items() if not (rc == 1 or rc < 0)}
    assert not survivors, f"mistakes no pin detects: {survivors}"
