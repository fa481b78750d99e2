"""Benchmark of one IT-MPC control iteration on GB300.

Workload (the working-size configuration): K = 2048 samples, T = 100 steps,
6->32->32->4 tanh dynamics network (Xavier, seed 42), 1024 x 1024 FP32
costmap at 0.1 m of a seeded closed spline track, speed target 6 m/s, 1e4
impulses, lambda = 1, sigma = (0.3, 0.35).  All inputs are synthetic.

A step is one full iteration (noise, rollouts, costs, weights, update) through
``itmpc_iterate``; the iteration index advances every step and U' is fed back
as the next nominal sequence.  L2 is flushed (256 MiB write) before every timed
step; only the iteration itself is inside each step's CUDA-event pair.

With N > 1 ranks (torchrun, one GPU each) a step is ONE iteration of N x 2048
samples, sharded over the ranks: rank r rolls out global samples
2048 r .. 2048 (r + 1) - 1 (``itmpc_iterate_shard``), the ranks all-gather their
partial records (NCCL; ``ITMPC_BENCH_BACKEND=gloo`` exchanges them through the
host instead) and every rank merges them on its GPU (``itmpc_merge_shards``):
weak scaling, 2048 samples per GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
paper ships no implementation to run).  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MPPI rollout-steps/s & control updates/s; BF16/batched vs FP32 at stated error"
UNIT = "rollout-steps/s"
K_WORK, T_WORK, H_WORK = 2048, 100, 32
FLOP_PER_SAMPLE_STEP = 2 * (6 * H_WORK + H_WORK * H_WORK + H_WORK * 4)  # network MACs x 2 = 2688
PROFILE = os.path.join(ROOT, "profiles", "iterate_fp32_K2048_T100.md")
KERNEL_SOURCES = ["paper_1707_02342_gb300/csrc/iterate_fp32.cu", "paper_1707_02342_gb300/csrc/itmpc_device.cuh",
                  "paper_1707_02342_gb300/csrc/itmpc_fused.cuh", "paper_1707_02342_gb300/csrc/itmpc_merge.cuh",
                  "paper_1707_02342_gb300/csrc/itmpc_sum.cuh"]


ADJ_PROFILE = os.path.join(ROOT, "profiles", "adj_backward_K4096_T100_H64.md")
ADJ_SOURCES = ["paper_1707_02342_gb300/csrc/iterate_adj.cu"]
# the forms' dominant kernels: (profile, the sources its hash covers)
FORM_PROFILES = {
    "batched": ("tps_rollout_batched256.md", ["iterate_tps.cu", "itmpc_units.cuh", "itmpc_sum.cuh"]),
    "fp32_h128": ("wide_rollout_H128_K16384.md", ["iterate_wide.cu"]),
    "bf16": ("tc_rollout_bf16_K16384.md", ["iterate_tc.cu", "itmpc_tcgen05.cuh"]),
    "fp8": ("tc_rollout_bf16_K16384.md", ["iterate_tc.cu", "itmpc_tcgen05.cuh"]),
    "update_from_noise": ("wsum_partial4_K776192_T100.md", ["wsum.cu"]),
}


def form_traffic(name: str):
    """DRAM bytes per launch of a form's dominant kernel from its committed ncu summary, or None."""
    prof, srcs = FORM_PROFILES[name]
    key = "traffic_bytes_per_launch_fp8" if name == "fp8" else "traffic_bytes_per_launch"
    return profiled_traffic(os.path.join(ROOT, "profiles", prof), [f"paper_1707_02342_gb300/csrc/{f}" for f in srcs],
                            key)


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha1()
    for f in sources or KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(profile=PROFILE, sources=None, key="traffic_bytes_per_launch"):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    if not os.path.exists(profile):
        return None
    text = open(profile).read()
    m_src = re.search(r"kernel_source_sha1[^:]*:\s*([0-9a-f]+)", text)
    m_b = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_src or not m_b or m_src.group(1) != kernel_source_hash(sources):
        return None
    return float(m_b.group(1))


def workload():
    from paper_1707_02342_gb300 import inputs

    tmap = inputs.track_costmap(inputs.spline_centerline(1), 1024, 0.1, 2.5)
    layers = inputs.mlp_xavier((6, H_WORK, H_WORK, 4), seed=42)
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 4.0
    U = inputs.nominal_controls(T_WORK, seed=9, scale=0.2)
    params = dict(dt=0.02, lam=1.0, gamma=0.0, alpha_explore=0.0, sigma=(0.3, 0.35), u_min=(-1.0, -1.0),
                  u_max=(1.0, 1.0), cost_w=(1.0, 1.0, 1.0, 1.0), v_des=6.0, crash_cost=1e4, crash_decay=0.9,
                  track_thresh=0.99, slip_thresh=0.75, map_cap=2.5, seed=0x170702342)
    return tmap, layers, x0, U, params


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(seconds: float = 10.0, min_iters: int = 2):
    """The FP64 oracle on the host cores: full iterations of the workload for about ``seconds``."""
    import numpy as np

    import oracle

    tmap, layers, x0, U, params = workload()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    P = oracle.Problem(K=K_WORK, T=T_WORK, layers=layers, costmap=tmap.data, res=tmap.res, origin_x=tmap.origin_x,
                       origin_y=tmap.origin_y, lam=params["lam"], sigma=params["sigma"], cost_w=params["cost_w"],
                       n_threads=cores)
    U64 = U.astype(np.float64)
    n, t0 = 0, time.perf_counter()
    while n < min_iters or time.perf_counter() - t0 < seconds:
        rc, U64, _, _ = oracle.iterate(P, x0, U64, n)
        n += 1
    dt = time.perf_counter() - t0
    # the same oracle on one host core, a few iterations
    P1 = P.replace(n_threads=1)
    U1 = U.astype(np.float64)
    n1, t1 = 0, time.perf_counter()
    while n1 < 1 or time.perf_counter() - t1 < min(3.0, seconds / 3):
        rc, U1, _, _ = oracle.iterate(P1, x0, U1, n1)
        n1 += 1
    d1 = time.perf_counter() - t1
    return {"value": K_WORK * T_WORK * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} full iterations of K={K_WORK}, T={T_WORK} (FP64 C oracle, OpenMP over samples) "
                      f"in {dt:.1f} s",
            "single_core": {"value": K_WORK * T_WORK * n1 / d1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} full iterations on one core in {d1:.1f} s"}}, dt / n


def measure_batched(params, layers, steps: int = 50, warmup: int = 10):
    """The batching form: 256 independent instances (K in {512..8192}, T in {40, 60, 100, 150},
    8 seeded 1024 x 1024 spline maps; instance table seed 7) in one itmpc_iterate_batch call."""
    import numpy as np
    import torch

    from paper_1707_02342_gb300 import inputs, itmpc

    Ks, Ts, ms = inputs.instance_table(256, seed=7)
    maps = [inputs.track_costmap(inputs.spline_centerline(seed), 1024, 0.1, 2.5) for seed in range(1, 9)]
    p = dict(params)
    ctl = itmpc.Controller(int(Ks.max()), int(Ts.max()), T_max=int(Ts.max()), hidden=H_WORK, **p)
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in maps], maps[0].res, maps[0].origin_x,
                     maps[0].origin_y)
    ctl.reserve_batch(256, int(Ks.sum()))
    insts = []
    for i, (K, T, m) in enumerate(zip(Ks, Ts, ms)):
        x0 = inputs.start_state(maps[m].centerline)
        x0[4] = 4.0
        U = torch.tensor(inputs.nominal_controls(int(T), seed=100 + i, scale=0.2), device="cuda")
        insts.append(dict(K=int(K), T=int(T), map_index=int(m), instance=i, iter=0,
                          x0=torch.tensor(x0, device="cuda"), U=U, U_out=U))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for it in range(warmup):
        for d in insts:
            d["iter"] = it
        ctl.iterate_batch(insts)
    torch.cuda.synchronize()
    assert ctl.read_status() == itmpc.OK
    # launch shape picked by the library's autotuner on this batch (outputs go to scratch)
    nt, ctas = ctl.autotune_batch(insts, reps=2)

    def timed(step):
        times = []
        for it in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(it)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        assert ctl.read_status() == itmpc.OK
        return float(np.mean(times))

    def direct(it):
        for d in insts:
            d["iter"] = warmup + it
        ctl.iterate_batch(insts)

    ms_direct = timed(direct)
    # closed loop as a CUDA graph: each replay advances every instance's iteration index on the device
    for d in insts:
        d["iter"] = warmup + steps
    ctl.batch_graph_create(insts)
    ctl.batch_graph_launch()
    torch.cuda.synchronize()
    ms_graph = timed(lambda it: ctl.batch_graph_launch())
    ctl.close()
    ms_per = ms_graph
    sample_steps = int((Ks.astype(np.int64) * Ts).sum())
    achieved = FLOP_PER_SAMPLE_STEP * sample_steps / (ms_per * 1e-3) / 1e12
    return {"workload": "256 instances, K~U{512..8192}, T~U{40,60,100,150}, 8 spline maps 1024^2, H=32 FP32",
            "sample_steps_per_launch": sample_steps, "ms_per_step": ms_per, "value": sample_steps / (ms_per * 1e-3),
            "unit": UNIT, "mode": "CUDA-graph replay (rollout, merge, iteration advance)",
            "ms_per_step_direct_call": ms_direct, "autotuned_tile": {"samples_per_unit": nt, "ctas_per_sm": ctas},
            "gpu_launches_per_step": 3, "achieved_tflops": achieved}


def _timed(fn, steps: int, warmup: int, flush):
    """Median and mean CUDA-event time (ms) of fn() over ``steps`` calls, L2 flushed before each."""
    import numpy as np
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts)), float(np.mean(ts))


def _controller(K, T, H, tmap, layers, params, **kw):
    import torch

    from paper_1707_02342_gb300 import itmpc

    ctl = itmpc.Controller(K, T, hidden=H, **dict(params, **kw))
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmap(torch.tensor(tmap.data, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    return ctl


def measure_precision(params, flush, steps: int = 50, warmup: int = 10):
    """The precision form: K = 16384, T = 100, 6->128->128->4 network, FP32 vs BF16 vs FP8 (tcgen05),
    each timed through itmpc_iterate.  Returns the JSON object and the GPU outputs (costs, weights, U')
    that the CPU-baseline leg compares with the FP64 oracle."""
    import torch

    from paper_1707_02342_gb300 import inputs, itmpc

    import numpy as np

    K, T, H = 16384, 100, 128
    tmap = inputs.track_costmap(inputs.spline_centerline(1), 1024, 0.1, 2.5)
    layers = inputs.mlp_xavier((6, H, H, 4), seed=42)
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 4.0
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    it = 5
    out = {"workload": f"it-mpc iteration K={K} T={T} 6->{H}->{H}->4 spline-1024 map",
           "sample_steps_per_launch": K * T}
    gpu = {}
    flop = 2 * (6 * H + H * H + 4 * H) * K * T
    x0_d, U_d = torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda")
    base_ms = None
    for name, prec in (("fp32", itmpc.FP32), ("bf16", itmpc.BF16), ("fp8", itmpc.FP8)):
        ctl = _controller(K, T, H, tmap, layers, params, precision=prec)
        Uo, w, S = torch.empty_like(U_d), torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
        med, mean = _timed(lambda: ctl.iterate(x0_d, U_d, it, Uo, w, S), steps, warmup, flush)
        assert ctl.read_status() == itmpc.OK
        gpu[name] = tuple(t.double().cpu().numpy() for t in (S, w, Uo))
        if name == "fp32":
            # the U' error budget: the Monte-Carlo spread of U' over 16 other noise draws (iteration
            # indices) of the same iteration, per element, from the FP32 form
            draws = []
            for j in range(16):
                ctl.iterate(x0_d, U_d, it + 1 + j, Uo, w, S)
                draws.append(Uo.double().cpu().numpy())
            mc_std = np.std(np.array(draws), axis=0, ddof=1)
            Uo.zero_()
            ctl.iterate(x0_d, U_d, it, Uo, w, S)  # leave this draw's outputs as measured above
            out["U_out_mc_std_l2"] = float(np.linalg.norm(mc_std))
        base_ms = base_ms or mean
        out[name] = {"ms_per_step": mean, "ms_median": med, "value": K * T / (mean * 1e-3), "unit": UNIT,
                     "speedup_vs_fp32": base_ms / mean, "algorithmic_tflops": flop / (mean * 1e-3) / 1e12,
                     "err_vs_fp64": None}
        ctl.close()
    case = {"K": K, "T": T, "layers": layers, "tmap": tmap, "x0": x0, "U": U, "it": it, "gpu": gpu}
    return out, case


def measure_adjoint(params, flush, steps: int = 50, warmup: int = 10, every: int = 10):
    """The adjoint form: K = 4096, T = 100, 6->64->64->4, checkpoints every 10 steps; forward + backward
    time next to the plain iteration and to central differences.  Returns the JSON object and the GPU
    gradients that the CPU-baseline leg compares with the FP64 oracle's."""
    import numpy as np
    import torch

    from paper_1707_02342_gb300 import inputs

    K, T, H = 4096, 100, 64
    tmap = inputs.track_costmap(inputs.spline_centerline(1), 1024, 0.1, 2.5)
    layers = inputs.mlp_xavier((6, H, H, 4), seed=42)
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 4.0
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    it = 11
    ctl = _controller(K, T, H, tmap, layers, params)
    ctl.reserve_adjoint()
    x0_d, U_d = torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda")
    ck = torch.empty(ctl.ckpt_floats(every), device="cuda")
    Uo, w, S, J = torch.empty_like(U_d), torch.empty(K, device="cuda"), torch.empty(K, device="cuda"), \
        torch.empty(1, device="cuda")
    gU_h = np.random.default_rng(3).standard_normal((T, 2)).astype(np.float32)
    gJ, gU = torch.ones(1, device="cuda"), torch.tensor(gU_h, device="cuda")
    nf = 12 * H + H * H + 4
    g_cw, g_U, g_net = torch.empty(4, device="cuda"), torch.empty_like(U_d), torch.empty(nf, device="cuda")
    plain = _timed(lambda: ctl.iterate(x0_d, U_d, it, Uo, w, S), steps, warmup, flush)[1]
    fwd = _timed(lambda: ctl.iterate_fwd(x0_d, U_d, it, every, ck, Uo, w, S, J), steps, warmup, flush)[1]
    bwd = _timed(lambda: ctl.iterate_bwd(U_d, it, every, ck, w, S, Uo, gJ, gU, g_cw, g_U, g_net), steps, warmup,
                 flush)[1]
    assert ctl.read_status() == 0
    active = int(np.count_nonzero(w.cpu().numpy()))
    case = {"K": K, "T": T, "layers": layers, "tmap": tmap, "x0": x0, "U": U, "it": it, "gU": gU_h,
            "S": S.double().cpu().numpy(),
            "gpu": {k: v.double().cpu().numpy().ravel() for k, v in (("cost_w", g_cw), ("U", g_U), ("net", g_net))}}
    ctl.close()
    n_params = nf + 4 + 2 * T
    bwd_flop = 2 * 2 * (6 * H + H * H + 4 * H) * active * T  # reverse network sweep: twice the forward MACs
    out = {"workload": f"adjoint of one iteration K={K} T={T} 6->{H}->{H}->4 spline-1024 map, "
                       f"checkpoints every {every} steps", "active_samples": active,
           "plain_ms": plain, "fwd_ms": fwd, "bwd_ms": bwd, "fwd_plus_bwd_over_plain": (fwd + bwd) / plain,
           "n_params": n_params,
           "speedup_vs_central_differences": 2 * n_params * plain / (fwd + bwd),
           "grad_rel_err_vs_fp64": None,
           "bwd_roofline": {"bound": "alu", "achieved": bwd_flop / (bwd * 1e-3) / 1e12, "unit": "TFLOP/s",
                            "algorithmic_flop": bwd_flop,
                            "traffic": profiled_traffic(ADJ_PROFILE, ADJ_SOURCES)}}
    return out, case


def fp64_error_reports(forms, cases, params, cores):
    """Part of the CPU-baseline leg: the FP64 oracle on the host cores computes the references of the
    precision and adjoint forms' error reports from the GPU outputs measured above."""
    import numpy as np

    import oracle

    def problem(c):
        return oracle.Problem(K=c["K"], T=c["T"], layers=c["layers"], costmap=c["tmap"].data, res=c["tmap"].res,
                              origin_x=c["tmap"].origin_x, origin_y=c["tmap"].origin_y, lam=params["lam"],
                              sigma=params["sigma"], cost_w=params["cost_w"], n_threads=cores)

    c = cases["precision"]
    t0 = time.perf_counter()
    rc, U64, w64, S64 = oracle.iterate(problem(c), c["x0"], c["U"], c["it"])
    forms["precision"]["oracle_s"] = time.perf_counter() - t0
    J64 = float(np.sum(w64[w64 > 0] * S64[w64 > 0]))
    for name, (Sg, wg, Ug) in c["gpu"].items():
        rel = np.abs(Sg - S64) / np.maximum(np.abs(S64), 1.0)
        Jg = float(np.sum(wg[wg > 0] * Sg[wg > 0]))
        forms["precision"][name]["err_vs_fp64"] = {
            "cost_rel_median": float(np.median(rel)), "cost_rel_p99": float(np.quantile(rel, 0.99)),
            "cost_rel_max": float(rel.max()), "expected_cost_rel": abs(Jg - J64) / abs(J64),
            "U_out_err_over_update": float(np.abs(Ug - U64).max() / np.abs(U64 - c["U"]).max()),
            # the budget: ||U'_form - U'_FP64||_2 <= the Monte-Carlo spread of U' (||std over draws||_2)
            "U_out_err_over_mc_std": float(np.linalg.norm(Ug - U64) / forms["precision"]["U_out_mc_std_l2"])}
    c = cases["adjoint"]
    ref = oracle.iterate_vjp(problem(c), c["x0"], c["U"], c["it"], 1.0, c["gU"].astype(np.float64), S_use=c["S"])
    want = {"cost_w": ref["g_cost_w"], "U": ref["g_U"], "net": ref["g_net"]}
    forms["adjoint"]["grad_rel_err_vs_fp64"] = {
        k: float(np.linalg.norm(c["gpu"][k] - want[k].ravel()) / np.linalg.norm(want[k])) for k in want}


def measure_closed_loop(tmap, layers, x0, U, params, flush, steps: int = 200, warmup: int = 10):
    """The closed loop of Alg. 1 at the working size: iteration, Savitzky-Golay smoothing, the first
    control through the noise-free model (the simulated plant) and the warm-start shift, as one CUDA
    graph replayed per control step (and as direct itmpc_control_step calls)."""
    import numpy as np
    import torch

    from paper_1707_02342_gb300 import itmpc

    ctl = _controller(K_WORK, T_WORK, H_WORK, tmap, layers, params)
    x = torch.tensor(x0, device="cuda")
    Ud = torch.tensor(U, device="cuda")
    ua = torch.empty(2, device="cuda")
    stream = torch.cuda.current_stream()
    it = [0]

    def direct():
        ctl.control_step(x, Ud, it[0], smoothing=itmpc.SMOOTH_SGF, plant=1, u_applied=ua)
        it[0] += 1

    ms_direct = _timed(direct, steps, warmup, flush)[1]
    x.copy_(torch.tensor(x0, device="cuda"))
    Ud.copy_(torch.tensor(U, device="cuda"))
    ctl.control_graph_create(x, Ud, 0, smoothing=itmpc.SMOOTH_SGF, plant=1, u_applied=ua)
    for _ in range(warmup):
        ctl.control_graph_launch()
    torch.cuda.synchronize()
    # steps back to back (no flush between them: a closed loop runs them back to back)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctl.control_graph_launch()
    b.record(stream)
    b.synchronize()
    ms_graph = a.elapsed_time(b) / steps
    assert ctl.read_status() == itmpc.OK
    xs = x.cpu().numpy()
    ctl.close()
    return {"workload": f"closed loop of Alg. 1, K={K_WORK} T={T_WORK} H={H_WORK} spline-1024 map: iteration, "
                        "SGF(U'), plant step, warm start", "ms_per_control_step": ms_graph,
            "control_updates_per_s": 1e3 / ms_graph, "rollout_steps_per_s": K_WORK * T_WORK / (ms_graph * 1e-3),
            "mode": f"CUDA graph, {steps} replays back to back", "ms_per_control_step_direct_calls": ms_direct,
            "gpu_launches_per_step": 2, "final_state_finite": bool(np.all(np.isfinite(xs)))}


def measure_cem(tmap, layers, x0, U, params, flush, steps: int = 200, warmup: int = 10, delta: float = 0.8):
    """Cross-entropy MPC (Alg. 3 weights, delta = 0.8 as in the paper's experiments) on the working
    workload, next to the information-theoretic iteration on the same rollouts."""
    import torch

    ctl = _controller(K_WORK, T_WORK, H_WORK, tmap, layers, params)
    x = torch.tensor(x0, device="cuda")
    Ud = torch.tensor(U, device="cuda")
    Uo, w, S = torch.empty_like(Ud), torch.empty(K_WORK, device="cuda"), torch.empty(K_WORK, device="cuda")
    ms_cem = _timed(lambda: ctl.iterate_cem(x, Ud, 3, delta, Uo, w, S), steps, warmup, flush)[1]
    ms_it = _timed(lambda: ctl.iterate(x, Ud, 3, Uo, w, S), steps, warmup, flush)[1]
    assert ctl.read_status() == 0
    ctl.close()
    return {"workload": f"cross-entropy MPC iteration K={K_WORK} T={T_WORK} H={H_WORK} spline-1024 map, "
                        f"delta={delta}", "ms_per_step": ms_cem, "ms_per_step_it_mpc": ms_it,
            "value": K_WORK * T_WORK / (ms_cem * 1e-3), "unit": UNIT, "gpu_launches_per_step": 3}


def measure_basis(tmap, params, flush, steps: int = 50, warmup: int = 10):
    """The basis-function dynamics model (25 basis functions, synthetic Theta, seed 5) on the working
    map, T = 100: one iteration at K = 2048 and at K = 65536 (thread-per-sample kernels)."""
    import torch

    from paper_1707_02342_gb300 import inputs, itmpc

    theta = torch.tensor(inputs.basis_theta(5), device="cuda")
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 4.0
    x = torch.tensor(x0, device="cuda")
    out = {"workload": "basis-function dynamics model, T=100, spline-1024 map, synthetic Theta (seed 5)"}
    for K in (K_WORK, 65536):
        ctl = itmpc.Controller(K, T_WORK, hidden=H_WORK, dynamics=itmpc.DYN_BASIS, **params)
        ctl.set_basis(theta)
        ctl.set_costmap(torch.tensor(tmap.data, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
        U = torch.tensor(inputs.nominal_controls(T_WORK, seed=9, scale=0.2), device="cuda")
        Uo, w, S = torch.empty_like(U), torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
        ms = _timed(lambda: ctl.iterate(x, U, 2, Uo, w, S), steps, warmup, flush)[1]
        assert ctl.read_status() == 0
        ctl.close()
        out[f"K{K}"] = {"ms_per_step": ms, "value": K * T_WORK / (ms * 1e-3), "unit": UNIT}
    return out


def measure_update_hbm(params, layers, flush, steps: int = 50, warmup: int = 10):
    """The control law from materialised noise (itmpc_update_from_noise), the HBM-bound form of the
    update: eps of the batched workload's size (K = 776192 samples x T = 100 steps, 621 MB) streamed
    once per call, weights from a real iteration on the working map."""
    import torch

    from paper_1707_02342_gb300 import inputs

    K, T = 776192, 100
    tmap = inputs.track_costmap(inputs.spline_centerline(1), 1024, 0.1, 2.5)
    ctl = _controller(K, T, H_WORK, tmap, layers, params)
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 4.0
    x = torch.tensor(x0, device="cuda")
    U = torch.tensor(inputs.nominal_controls(T, seed=9, scale=0.2), device="cuda")
    Uo, w, S = torch.empty_like(U), torch.empty(K, device="cuda"), torch.empty(K, device="cuda")
    ctl.iterate(x, U, 3, Uo, w, S)
    eps = torch.empty((K, T, 2), device="cuda")
    ctl.noise(3, eps)
    U2 = torch.empty_like(U)
    med, mean = _timed(lambda: ctl.update_from_noise(eps, w, U, U2), steps, warmup, flush)
    # streamed: calls back to back between two events on the launching stream; eps is 4.8x the
    # L2, so every call reads it from HBM without a flush (host launch latency overlapped)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        ctl.update_from_noise(eps, w, U, U2)
    b.record(stream)
    b.synchronize()
    streamed = a.elapsed_time(b) / steps
    assert ctl.read_status() == 0
    err = float((U2 - Uo).abs().max())
    ctl.close()
    nbytes = K * T * 8 + 2 * K * 4 + 3 * 2 * T * 4  # eps once, weights twice, U / records / U'
    return {"workload": f"U' = sum_k w_k v_k from materialised noise, K={K} T={T} ({K * T * 8 / 1e6:.0f} MB)",
            "ms_per_call": streamed, "ms_per_call_isolated": mean, "ms_median_isolated": med,
            "timing": f"{steps} calls back to back (eps larger than L2, no flush); isolated: one call between "
                      "events, L2 flushed before each",
            "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (streamed * 1e-3) / 1e9,
            "achieved_gbs_isolated": nbytes / (mean * 1e-3) / 1e9, "max_abs_diff_vs_fused_update": err,
            "gpu_launches_per_call": 2}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    return d


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = max(1, args.steps)
    per = None
    import numpy as np

    import oracle

    tmap, layers, x0, U, params = workload()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    K_total = world * K_WORK  # the same iteration as the GPU arm's (N x 2048 samples sharded over N GPUs)
    P = oracle.Problem(K=K_total, T=T_WORK, layers=layers, costmap=tmap.data, res=tmap.res, origin_x=tmap.origin_x,
                       origin_y=tmap.origin_y, lam=params["lam"], sigma=params["sigma"], cost_w=params["cost_w"],
                       n_threads=cores)
    U64 = U.astype(np.float64)
    for i in range(args.warmup):
        _, U64, _, _ = oracle.iterate(P, x0, U64, i)
    # bounded: at most ~60 s of timed oracle work whatever --steps says
    t0 = time.perf_counter()
    n = 0
    for i in range(steps):
        _, U64, _, _ = oracle.iterate(P, x0, U64, args.warmup + i)
        n += 1
        if time.perf_counter() - t0 > 60.0:
            break
    dt = time.perf_counter() - t0
    per = dt / n
    value = K_total * T_WORK / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"it-mpc iteration K={K_total} T={T_WORK} H={H_WORK} spline-1024 map",
                       "K": K_total, "K_per_gpu": K_WORK, "T": T_WORK, "hidden": H_WORK, "map": "1024x1024@0.1m"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} full iterations (FP64 C oracle, OpenMP over samples)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "control_updates_per_s": 1.0 / per}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, world: int) -> float:
    """The largest value of x over the ranks (x itself on one rank)."""
    if world == 1:
        return x
    import torch

    dist = torch.distributed
    t = torch.tensor([x], dtype=torch.float64)
    if dist.get_backend() != "gloo":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1707_02342_gb300 import build as nbuild
    from paper_1707_02342_gb300 import itmpc

    dev = local_rank % torch.cuda.device_count()
    torch.cuda.set_device(dev)
    if rank == 0:
        nbuild.build()
    if world > 1:
        torch.distributed.barrier()
    tmap, layers, x0, U, params = workload()
    stream = torch.cuda.current_stream()
    # N > 1: every rank holds a shard of one iteration (same noise stream, instance tag 0)
    ctl = itmpc.Controller(K_WORK, T_WORK, hidden=H_WORK, instance=0, **params)
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmap(torch.tensor(tmap.data, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    x0_d = torch.tensor(x0, device="cuda")
    U0_d = torch.tensor(U, device="cuda")
    U_d = U0_d.clone()
    w_d = torch.empty(K_WORK, device="cuda")
    S_d = torch.empty(K_WORK, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    launches_per_step = 1 if K_WORK <= 16384 else 2
    K_total = world * K_WORK
    if world > 1:
        dist = torch.distributed
        gloo = dist.get_backend() == "gloo"
        stride = itmpc.partial_stride(T_WORK)
        rec_me = torch.zeros(stride, device="cuda")
        rec_all = torch.zeros((world, stride), device="cuda")
        launches_per_step = 2  # the shard's iteration kernel and the record merge

        def exchange():
            if gloo:  # through the host (one GPU can carry several ranks this way)
                parts = [torch.zeros(stride) for _ in range(world)]
                dist.all_gather(parts, rec_me.cpu())
                rec_all.copy_(torch.stack(parts))
            else:
                dist.all_gather_into_tensor(rec_all.view(-1), rec_me)

        def step(i):
            ctl.iterate_shard(x0_d, U_d, i, rank * K_WORK, K_total, rec_me, S_d)
            exchange()
            ctl.merge_shards(rec_all, K_total, U_d, U_d, S_d, w_d)
    else:
        def step(i):
            ctl.iterate(x0_d, U_d, i, U_d, w_d, S_d)

    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    assert ctl.read_status() == itmpc.OK
    U_d.copy_(U0_d)

    n = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    sampler = ClockSampler(dev)
    with sampler:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(n):
            flush.zero_()
            starts[i].record(stream)
            step(args.warmup + i)
            ends[i].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t_wall = time.perf_counter() - t_wall
    assert ctl.read_status() == itmpc.OK
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    mean_ms = max_over_ranks(float(step_ms.mean()), world)

    # end to end: h2d of x0 + U from pinned host memory, the step, d2h of U'
    e2e_n = min(n, 500)
    e2e_warm = max(10, args.warmup)
    if world == 1:
        # through the host-pointer entry point; the first call captures the context's host graph
        # (as every call after a parameter change would), so untimed calls come first
        x0_h = torch.tensor(x0).pin_memory().numpy()
        U_h = torch.tensor(U).pin_memory().numpy()
        Uo_h = torch.empty((T_WORK, 2), dtype=torch.float32).pin_memory().numpy()
        for i in range(e2e_warm):
            st = ctl.iterate_host(x0_h, U_h, i, Uo_h)
            assert st == itmpc.OK
        e2e_s = []
        for i in range(e2e_n):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctl.iterate_host(x0_h, U_h, args.warmup + i, Uo_h)
            e2e_s.append(time.perf_counter() - t0)
            assert st == itmpc.OK
            U_h[:] = Uo_h
        e2e_entry = "itmpc_iterate_host (pinned host buffers; includes copies and stream sync)"
    else:
        x0_p = torch.tensor(x0).pin_memory()
        U_p = torch.tensor(U).pin_memory()
        Uo_p = torch.empty((T_WORK, 2), dtype=torch.float32).pin_memory()

        def e2e_step(i):
            x0_d.copy_(x0_p, non_blocking=True)
            U_d.copy_(U_p, non_blocking=True)
            step(i)
            Uo_p.copy_(U_d, non_blocking=True)
            torch.cuda.synchronize()
            U_p.copy_(Uo_p)

        for i in range(e2e_warm):
            e2e_step(i)
        e2e_s = []
        for i in range(e2e_n):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(args.warmup + i)
            e2e_s.append(time.perf_counter() - t0)
        e2e_entry = ("itmpc_iterate_shard + record all-gather + itmpc_merge_shards with pinned-host copies of "
                     "x0, U in and U' out (torch.cuda copies; includes the stream sync)")
    e2e_med = float(np.median(e2e_s))
    e2e_mean = max_over_ranks(float(np.mean(e2e_s)), world)

    if rank != 0:
        return
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    sm_max = pk.get("sm_max_mhz", 2070.0)
    peak_tflops = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = FLOP_PER_SAMPLE_STEP * K_WORK * T_WORK / (float(step_ms.mean()) * 1e-3) / 1e12
    traffic = profiled_traffic()
    clocks = sampler.summary()
    value = world * K_WORK * T_WORK / (mean_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"it-mpc iteration K={K_total} T={T_WORK} H={H_WORK} spline-1024 map",
                   "K": K_total, "K_per_gpu": K_WORK, "T": T_WORK, "hidden": H_WORK, "map": "1024x1024@0.1m",
                   "crash_cost": 1e4,
                   "l2": "flushed before every timed step (256 MiB write, outside the step's events)",
                   "parallelism": ("one GPU" if world == 1 else
                                   f"K-sharded: one iteration of {K_total} samples over {world} GPUs, "
                                   f"{K_WORK} each; one all-gather of the {4 * itmpc.partial_stride(T_WORK)}-byte "
                                   f"partial records per iteration, then the log-sum-exp merge on every GPU")},
        "control_updates_per_s": world / (mean_ms * 1e-3),
        "ms_per_step_median": float(np.median(step_ms)),
        "wall_s_timed_region_incl_flush": t_wall,
        "e2e": {"value": world * K_WORK * T_WORK / e2e_mean, "unit": UNIT, "h2d_bytes_per_step": 4 * (7 + 2 * T_WORK),
                "d2h_bytes_per_step": 4 * 2 * T_WORK, "steps": e2e_n, "warmup": e2e_warm,
                "us_per_call_mean": e2e_mean * 1e6, "us_per_call_median": e2e_med * 1e6,
                "entry_point": e2e_entry},
        "gpu_launches": n * launches_per_step,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "iterate_fp32_kernel<32, 7, 2> (fused noise, rollout, cost, weights, update)",
                     "peak_derivation": f"{n_sm} SMs x 128 FP32 lanes x 2 FLOP x {sm_max:.0f} MHz (max SM clock)",
                     "algorithmic_flop_per_launch": FLOP_PER_SAMPLE_STEP * K_WORK * T_WORK},
        "clocks": clocks,
    }
    if world == 1 and not args.no_forms:
        bt = measure_batched(params, layers)
        bt["roofline"] = {"bound": "alu", "achieved": bt.pop("achieved_tflops"), "peak": peak_tflops,
                          "unit": "TFLOP/s"}
        bt["roofline"]["frac"] = bt["roofline"]["achieved"] / peak_tflops
        bt["roofline"]["traffic"] = form_traffic("batched")
        line["forms"] = {"batched": bt}
        pr, pr_case = measure_precision(params, flush)
        bf_peak = pk.get("bf16_tflops", 1900.0)
        for name, pkv in (("bf16", bf_peak), ("fp8", 2 * bf_peak)):
            pr[name]["roofline"] = {"bound": "tensor", "achieved": pr[name]["algorithmic_tflops"], "peak": pkv,
                                    "unit": "TFLOP/s", "frac": pr[name]["algorithmic_tflops"] / pkv,
                                    "peak_note": "measured bf16 burst" + (" x 2 (nominal fp8/bf16 ratio)"
                                                                           if name == "fp8" else ""),
                                    "traffic": form_traffic(name)}
        pr["fp32"]["roofline"] = {"bound": "alu", "achieved": pr["fp32"]["algorithmic_tflops"], "peak": peak_tflops,
                                  "unit": "TFLOP/s", "frac": pr["fp32"]["algorithmic_tflops"] / peak_tflops,
                                  "traffic": form_traffic("fp32_h128")}
        line["forms"]["precision"] = pr
        line["forms"]["closed_loop"] = measure_closed_loop(tmap, layers, x0, U, params, flush)
        line["forms"]["cem"] = measure_cem(tmap, layers, x0, U, params, flush)
        line["forms"]["basis"] = measure_basis(tmap, params, flush)
        uh = measure_update_hbm(params, layers, flush)
        hbm = pk.get("hbm_gbs", 6800.0)
        uh["roofline"] = {"bound": "hbm", "achieved": uh["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                          "frac": uh["achieved_gbs"] / hbm, "peak_note": "measured copy bandwidth",
                          "traffic": form_traffic("update_from_noise")}
        line["forms"]["update_from_noise"] = uh
        ad, ad_case = measure_adjoint(params, flush)
        ad["bwd_roofline"]["peak"] = peak_tflops
        ad["bwd_roofline"]["frac"] = ad["bwd_roofline"]["achieved"] / peak_tflops
        line["forms"]["adjoint"] = ad
    if world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_oracle_rate(seconds=args.cpu_seconds)
        line["cpu_baseline"] = cb
        if "forms" in line:
            cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
            fp64_error_reports(line["forms"], {"precision": pr_case, "adjoint": ad_case}, params, cores)
            cb["also"] = "FP64 references of the precision and adjoint forms' error reports"
    elif "forms" in line:
        line["forms"]["error_reports"] = "skipped with the CPU-baseline leg (--no-cpu-baseline)"
    print(json.dumps(line), flush=True)
    ctl.close()


def run_only(args):
    """One form alone, a few steps (for ncu captures of its kernels)."""
    import torch

    from paper_1707_02342_gb300 import build as nbuild

    torch.cuda.set_device(0)
    nbuild.build()
    tmap, layers, x0, U, params = workload()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    steps, warm = max(1, args.steps), args.warmup
    if args.only == "batched":
        out = measure_batched(params, layers, steps=steps, warmup=warm)
    elif args.only == "precision":
        out, _ = measure_precision(params, flush, steps=steps, warmup=warm)
    elif args.only == "update_from_noise":
        out = measure_update_hbm(params, layers, flush, steps=steps, warmup=warm)
    elif args.only == "basis":
        out = measure_basis(tmap, params, flush, steps=steps, warmup=warm)
    elif args.only == "cem":
        out = measure_cem(tmap, layers, x0, U, params, flush, steps=steps, warmup=warm)
    elif args.only == "closed_loop":
        out = measure_closed_loop(tmap, layers, x0, U, params, flush, steps=steps, warmup=warm)
    else:
        out, _ = measure_adjoint(params, flush, steps=steps, warmup=warm)
    print(json.dumps({"only": args.only, **out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / precision / adjoint forms")
    ap.add_argument("--only", choices=["batched", "precision", "adjoint", "closed_loop", "cem", "basis", "update_from_noise"], default=None,
                    help="run one form alone and print its JSON (profiling runs); not a benchmark line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.only:
        run_only(args)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank % torch.cuda.device_count())
        torch.distributed.init_process_group(os.environ.get("ITMPC_BENCH_BACKEND", "nccl"))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
