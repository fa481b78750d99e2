"""GPU parity of the batched form: many independent instances in one launch
(thread-per-sample kernels), against the FP64 oracle instance by instance.

Same tolerances as test_gpu_parity: costs within 1e-5 relative (samples that
pass within 2e-4 of an impulse threshold are counted and excused), weights and
U' within 1e-5 when the oracle recomputes them from the GPU's own costs.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_parity import check_costs, check_stagewise, oracle_for

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def two_ellipses():
    a = problems.ellipse_map()
    b = inputs.track_costmap(inputs.ellipse_centerline(17.0, 14.0), 512, 0.1, 2.0)
    return a, b


def run_batch(params, maps, layers, specs, T_max):
    """specs: list of dict(K, T, map, instance, iter, speed, useed). Returns per-instance numpy results."""
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc
    from tests import native

    native.load()
    p = dict(params)
    p.pop("K"), p.pop("T")
    K_max = max(s["K"] for s in specs)
    ctl = itmpc.Controller(K_max, T_max, T_max=T_max, hidden=32, **p)
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in maps], maps[0].res, maps[0].origin_x,
                     maps[0].origin_y)
    ctl.reserve_batch(len(specs), sum(s["K"] for s in specs))
    insts, keep = [], []
    for s in specs:
        x0 = problems.x0_for(maps[s["map"]], speed=s.get("speed", 3.0))
        U = inputs.nominal_controls(s["T"], seed=s.get("useed", 1), scale=0.2)
        d = dict(K=s["K"], T=s["T"], map_index=s["map"], instance=s["instance"], iter=s["iter"],
                 x0=torch.tensor(x0, device="cuda"), U=torch.tensor(U, device="cuda"))
        d["U_out"] = torch.empty_like(d["U"])
        d["weights"] = torch.empty(s["K"], device="cuda")
        d["costs"] = torch.empty(s["K"], device="cuda")
        d["stats"] = torch.empty(8, device="cuda")
        insts.append(d)
        keep.append((x0, U))
    ctl.iterate_batch(insts)
    st = ctl.read_status()
    out = []
    for d, (x0, U) in zip(insts, keep):
        out.append(dict(x0=x0, U=U, Uo=d["U_out"].double().cpu().numpy(), w=d["weights"].double().cpu().numpy(),
                        S=d["costs"].double().cpu().numpy(), stats=d["stats"].cpu().numpy()))
    ctl.close()
    return st, out


def test_small_batch_matches_oracle():
    maps = two_ellipses()
    layers = problems.network(32)
    params = problems.params_small()
    specs = [dict(K=37, T=13, map=0, instance=1, iter=4), dict(K=128, T=40, map=1, instance=2, iter=4),
             dict(K=300, T=7, map=0, instance=3, iter=9, speed=5.0), dict(K=129, T=25, map=1, instance=4, iter=1),
             dict(K=1, T=3, map=0, instance=5, iter=2), dict(K=200, T=64, map=1, instance=6, iter=3, useed=7)]
    st, out = run_batch(params, maps, layers, specs, T_max=64)
    assert st == 0
    for s, r in zip(specs, out):
        prm = dict(params, K=s["K"], T=s["T"], instance=s["instance"])
        P = oracle_for(prm, maps[s["map"]], layers)
        S_ref, _ = oracle.rollout_many(P, r["x0"], r["U"], s["iter"])
        check_costs(r["S"], S_ref)
        check_stagewise(P, s["iter"], r["U"], r["Uo"], r["w"], r["S"], params["sigma"])
        assert r["stats"][0] == pytest.approx(r["S"].min(), rel=1e-6)


def test_batch_agrees_with_single_instance_path():
    maps = two_ellipses()
    layers = problems.network(32)
    params = problems.params_working(K=512, T=50)
    spec = dict(K=512, T=50, map=0, instance=0, iter=21, speed=4.0, useed=3)
    st, out = run_batch(params, maps, layers, [spec], T_max=50)
    assert st == 0
    ctl = G.controller(params, maps[0], layers)
    Uo, w, S, st2 = G.run(ctl, out[0]["x0"], out[0]["U"], 21)
    assert st2 == 0
    near = np.zeros(512, bool)
    P = oracle_for(params, maps[0], layers)
    _, margins = oracle.rollout_many(P, out[0]["x0"], out[0]["U"], 21)
    near = margins < 2e-4
    ok = np.abs(out[0]["S"] - S) <= 2e-5 * np.maximum(np.abs(S), 1.0)
    assert np.all(ok | near)


@functools.lru_cache(maxsize=None)
def spline_maps(n=8):
    return tuple(problems.spline_map(seed) for seed in range(1, n + 1))


def test_full_size_batch_sampled_parity():
    """256 instances, K in {512..8192}, T in {40..150}, 8 seeded spline maps (instance table seed 7)."""
    Ks, Ts, ms = inputs.instance_table(256, seed=7)
    maps = spline_maps()
    layers = problems.network(32)
    params = problems.params_working()
    specs = [dict(K=int(K), T=int(T), map=int(m), instance=i, iter=5, speed=4.0, useed=100 + i)
             for i, (K, T, m) in enumerate(zip(Ks, Ts, ms))]
    st, out = run_batch(params, maps, layers, specs, T_max=150)
    assert st == 0
    rng = np.random.default_rng(4)
    for i in [0, 1, 17, 100, 255] + list(rng.choice(256, 3, replace=False)):
        s, r = specs[i], out[i]
        prm = dict(params, K=s["K"], T=s["T"], instance=s["instance"])
        P = oracle_for(prm, maps[s["map"]], layers)
        ks = rng.choice(s["K"], size=min(24, s["K"]), replace=False)
        S_ref, margins = oracle.rollout_many(P, r["x0"], r["U"], s["iter"], ks)
        check_costs(r["S"][ks], S_ref, margins)
        check_stagewise(P, s["iter"], r["U"], r["Uo"], r["w"], r["S"], params["sigma"])


def _batch_controller(params, maps, layers, specs, T_max, precision=0):
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc
    from tests import native

    native.load()
    p = dict(params, precision=precision)
    p.pop("K"), p.pop("T")
    H = layers[0][0].shape[0]
    ctl = itmpc.Controller(max(s["K"] for s in specs), T_max, T_max=T_max, hidden=H, **p)
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in maps], maps[0].res, maps[0].origin_x,
                     maps[0].origin_y)
    ctl.reserve_batch(len(specs), sum(s["K"] for s in specs))
    insts = []
    for s in specs:
        x0 = problems.x0_for(maps[s["map"]], speed=s.get("speed", 3.0))
        U = inputs.nominal_controls(s["T"], seed=s.get("useed", 1), scale=0.2)
        insts.append(dict(K=s["K"], T=s["T"], map_index=s["map"], instance=s["instance"], iter=s["iter"],
                          x0=torch.tensor(x0, device="cuda"), U=torch.tensor(U, device="cuda"),
                          costs=torch.empty(s["K"], device="cuda"), weights=torch.empty(s["K"], device="cuda")))
    return ctl, insts


SPECS = [dict(K=37, T=13, map=0, instance=1, iter=4), dict(K=700, T=40, map=1, instance=2, iter=4),
         dict(K=300, T=7, map=0, instance=3, iter=9, speed=5.0), dict(K=129, T=25, map=1, instance=4, iter=1),
         dict(K=1, T=3, map=0, instance=5, iter=2)]


def test_autotune_keeps_costs_and_caller_buffers():
    """Every candidate tile gives bit-identical costs (samples are independent); the weights and U' only
    change by the merge's summation order; tuning never writes the caller's outputs."""
    torch = G.torch_cuda()
    maps = two_ellipses()
    layers = problems.network(32)
    ctl, insts = _batch_controller(problems.params_small(), maps, layers, SPECS, T_max=64)
    for d in insts:
        d["U_out"] = torch.empty_like(d["U"])
    ctl.iterate_batch(insts)
    assert ctl.read_status() == 0
    ref = [(d["costs"].clone(), d["weights"].clone(), d["U_out"].clone()) for d in insts]
    for d in insts:
        d["costs"].fill_(-1.0)
        d["U_out"].fill_(-1.0)
    nt, ctas = ctl.autotune_batch(insts, reps=1)
    assert nt in (64, 128, 256) and ctas >= 0
    torch.cuda.synchronize()
    for d in insts:
        assert bool((d["costs"] == -1.0).all()) and bool((d["U_out"] == -1.0).all())
    ctl.iterate_batch(insts)
    assert ctl.read_status() == 0
    for d, (S, w, Uo) in zip(insts, ref):
        assert torch.equal(d["costs"], S)
        torch.testing.assert_close(d["weights"], w, rtol=0, atol=1e-6 * float(w.max()))
        torch.testing.assert_close(d["U_out"], Uo, rtol=0, atol=1e-6)
    ctl.close()


@pytest.mark.parametrize("precision,H", [(0, 32), (1, 128)])
def test_graph_replay_equals_sequential_iterations(precision, H):
    """Closed loop in a CUDA graph: replay r draws iteration iter + r and starts from the previous U'."""
    torch = G.torch_cuda()
    maps = two_ellipses()
    layers = problems.network(H)
    params = problems.params_small()
    ctl, insts = _batch_controller(params, maps, layers, SPECS, T_max=64, precision=precision)
    U0 = [d["U"].clone() for d in insts]
    # sequential reference: three iterate_batch calls, U' fed back, iter advanced by hand
    seq = [dict(d, U=u.clone()) for d, u in zip(insts, U0)]
    for d in seq:
        d["U_out"] = d["U"]
    for r in range(3):
        for d, s in zip(seq, SPECS):
            d["iter"] = s["iter"] + r
        ctl.iterate_batch(seq)
        assert ctl.read_status() == 0
    want = [(d["U"].clone(), d["costs"].clone()) for d in seq]
    # the same through a captured graph, replayed three times
    gr = [dict(d, U=u.clone(), costs=torch.empty_like(d["costs"])) for d, u in zip(insts, U0)]
    for d in gr:
        d["U_out"] = d["U"]
    ctl.batch_graph_create(gr)
    for _ in range(3):
        ctl.batch_graph_launch()
    assert ctl.read_status() == 0
    for d, (U, S) in zip(gr, want):
        assert torch.equal(d["U"], U)
        assert torch.equal(d["costs"], S)
    ctl.batch_graph_destroy()
    with pytest.raises(Exception):
        ctl.batch_graph_launch()
    ctl.close()
