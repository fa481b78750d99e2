"""Sample-sharded iteration on the GPU: itmpc_iterate_shard + record merge.

A K_total-sample iteration runs as several contexts, each owning a contiguous
range of global sample indices; each writes its partial record (Alg. 2's
log-sum-exp reduction shifted by the shard's own minimum) and the records are
merged (itmpc_merge_partials on the host, itmpc_merge_shards on the device).
The noise of a sample is Philox of its global index, so the shards draw the
unsharded iteration's samples:
  * shards that run the same kernel as the unsharded context give the same
    costs bit for bit; other kernels within 1e-5 relative (the parity bound);
  * the merged U' equals the unsharded GPU U' to a few FP32 roundings, and the
    oracle's Alg. 2 and control law applied to the shards' costs within 1e-5;
  * the exploration split of Alg. 1 counts global samples (alpha > 0).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs, itmpc
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu

REL = 1e-5


def _workload(K_total, T, H=32, **kw):
    tmap = problems.spline_map(1)
    layers = problems.network(H)
    params = problems.params_working(K=K_total, T=T, **kw)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    return tmap, layers, params, x0, U


def _shards(torch, tmap, layers, params, x0, U, it, sizes):
    """Run one shard context per size; returns (records (n x stride) tensor, costs list, contexts)."""
    K_total, T = params["K"], params["T"]
    stride = itmpc.partial_stride(T)
    recs = torch.zeros((len(sizes), stride), device="cuda")
    x0_d, U_d = torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda")
    costs, ctls, k_base = [], [], 0
    for i, n in enumerate(sizes):
        ctl = G.controller(dict(params, K=n), tmap, layers)
        S = torch.empty(n, device="cuda")
        ctl.iterate_shard(x0_d, U_d, it, k_base, K_total, recs[i], S)
        costs.append(S)
        ctls.append(ctl)
        k_base += n
    assert k_base == K_total
    torch.cuda.synchronize()
    return recs, costs, ctls


def _check_merged(P, it, U, Uo, S_all, Uo_unsharded, tol_vs_gpu):
    scale = max(np.abs(Uo_unsharded).max(), 0.35)
    np.testing.assert_allclose(Uo, Uo_unsharded, rtol=0, atol=tol_vs_gpu * scale)
    rc, w_ref, _, _ = oracle.weights(S_all, P.lam)
    assert rc == 0
    U_ref = oracle.update(P, it, w_ref, U)
    np.testing.assert_allclose(Uo, U_ref, rtol=0, atol=REL * max(np.abs(U_ref).max(), 0.35))
    return w_ref


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_two_equal_shards_match_the_unsharded_iteration(alpha):
    torch = G.torch_cuda()
    it = 7
    tmap, layers, params, x0, U = _workload(2048, 100, alpha_explore=alpha)
    ctl = G.controller(params, tmap, layers)
    Uo_g, w_g, S_g, st = G.run(ctl, x0, U, it)
    assert st == 0
    recs, costs, ctls = _shards(torch, tmap, layers, params, x0, U, it, [1024, 1024])
    S_sh = np.concatenate([c.double().cpu().numpy() for c in costs])
    # the same fused kernel: every sample's arithmetic is the same, whatever the launch shape
    np.testing.assert_array_equal(S_sh, S_g)
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    # host merge
    st, Uo_h = itmpc.merge_partials(recs.cpu().numpy(), U, params["lam"])
    assert st == 0
    _check_merged(P, it, U, Uo_h.astype(np.float64), S_sh, Uo_g, 2e-6)
    # device merge on shard 0, with shard 0's weights under the global normaliser
    U_d = torch.tensor(U, device="cuda")
    Uo_d, w0 = torch.empty_like(U_d), torch.empty(1024, device="cuda")
    ctls[0].merge_shards(recs, 2048, U_d, Uo_d, costs[0], w0)
    assert ctls[0].read_status() == 0
    w_ref = _check_merged(P, it, U, Uo_d.double().cpu().numpy(), S_sh, Uo_g, 2e-6)
    np.testing.assert_allclose(w0.double().cpu().numpy(), w_ref[:1024], rtol=0, atol=REL * w_ref.max())
    np.testing.assert_allclose(w0.double().cpu().numpy(), w_g[:1024], rtol=0, atol=1e-6 * w_g.max())
    stats = ctls[0].stats()
    assert stats[0] == pytest.approx(S_g.min(), rel=1e-7)
    assert stats[4] == 2048
    for c in ctls + [ctl]:
        c.close()


def test_uneven_shards_on_different_kernels():
    """700 samples on the fused kernel, 4300 on the thread-per-sample kernel (K >= 4096)."""
    torch = G.torch_cuda()
    it = 3
    tmap, layers, params, x0, U = _workload(5000, 60, alpha_explore=0.1)
    ctl = G.controller(params, tmap, layers)
    Uo_g, w_g, S_g, st = G.run(ctl, x0, U, it)
    assert st == 0
    recs, costs, ctls = _shards(torch, tmap, layers, params, x0, U, it, [700, 4300])
    S_sh = np.concatenate([c.double().cpu().numpy() for c in costs])
    np.testing.assert_array_equal(S_sh[700:], S_g[700:])  # the same thread-per-sample kernel
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    S_ref, margins = oracle.rollout_many(P, x0, U, it, np.arange(700))
    ok = (np.abs(S_sh[:700] - S_ref) <= REL * np.maximum(np.abs(S_ref), 1.0)) | (margins < 2e-4)
    assert ok.all()
    st, Uo_h = itmpc.merge_partials(recs.cpu().numpy(), U, params["lam"])
    assert st == 0
    rc, w_ref, _, _ = oracle.weights(S_sh, P.lam)
    U_ref = oracle.update(P, it, w_ref, U)
    np.testing.assert_allclose(Uo_h, U_ref, rtol=0, atol=REL * max(np.abs(U_ref).max(), 0.35))
    for c in ctls + [ctl]:
        c.close()


@pytest.mark.parametrize("precision", [itmpc.BF16, itmpc.FP8])
def test_tensor_core_shards_match_unsharded(precision):
    """Shards on 128-sample boundaries hold the same MMA tiles as the unsharded launch."""
    torch = G.torch_cuda()
    it = 5
    tmap, layers, params, x0, U = _workload(512, 40, H=128, precision=precision)
    ctl = G.controller(params, tmap, layers)
    Uo_g, w_g, S_g, st = G.run(ctl, x0, U, it)
    assert st == 0
    recs, costs, ctls = _shards(torch, tmap, layers, params, x0, U, it, [128, 384])
    S_sh = np.concatenate([c.double().cpu().numpy() for c in costs])
    np.testing.assert_array_equal(S_sh, S_g)
    U_d = torch.tensor(U, device="cuda")
    Uo_d = torch.empty_like(U_d)
    ctls[1].merge_shards(recs, 512, U_d, Uo_d)
    scale = max(np.abs(Uo_g).max(), 0.35)
    np.testing.assert_allclose(Uo_d.double().cpu().numpy(), Uo_g, rtol=0, atol=2e-6 * scale)
    for c in ctls + [ctl]:
        c.close()


def test_shard_merge_nonfinite_and_argument_checks():
    torch = G.torch_cuda()
    tmap, layers, params, x0, U = _workload(256, 20)
    ctl = G.controller(dict(params, K=128), tmap, layers)
    x0_d, U_d = torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda")
    rec = torch.zeros((2, itmpc.partial_stride(20)), device="cuda")
    for k_base, K_total in [(-1, 256), (200, 256), (0, 100), (0, 2 ** 31)]:
        with pytest.raises(itmpc.ItmpcError):
            ctl.iterate_shard(x0_d, U_d, 0, k_base, K_total, rec[0])
    # records with no finite cost: U' = U and the status says so
    rec[:, 0] = float("inf")
    Uo = torch.empty_like(U_d)
    ctl.merge_shards(rec, 256, U_d, Uo)
    assert ctl.read_status() == itmpc.ERR_NONFINITE
    np.testing.assert_array_equal(Uo.cpu().numpy(), U_d.cpu().numpy())
    ctl.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, out_path):
    """One rank: its shard on cuda:0 through the library, records exchanged over gloo."""
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    it, K_total, T = 12, 3000, 80
    tmap, layers, params, x0, U = _workload(K_total, T, alpha_explore=0.2)
    bounds = [0, 1300, K_total]
    n = bounds[rank + 1] - bounds[rank]
    ctl = G.controller(dict(params, K=n), tmap, layers)
    rec = torch.zeros(itmpc.partial_stride(T), device="cuda")
    S = torch.empty(n, device="cuda")
    ctl.iterate_shard(torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda"), it, bounds[rank], K_total,
                      rec, S)
    torch.cuda.synchronize()
    recs = [torch.zeros(rec.numel()) for _ in range(world)]
    dist.all_gather(recs, rec.cpu())
    S_all = torch.zeros(K_total)  # every rank's costs in its own range, zeros elsewhere: a sum is exact
    S_all[bounds[rank]:bounds[rank + 1]] = S.cpu()
    dist.all_reduce(S_all)
    st, Uo = itmpc.merge_partials(torch.stack(recs).numpy(), U, params["lam"])
    if rank == 0:
        np.savez(out_path, Uo=Uo, S=S_all.numpy(), st=st)
    ctl.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_library_records(tmp_path):
    """Two processes, each with its shard context on cuda:0 (no kernel waits on another process),
    all-gather the records the library wrote and merge them; rank 0's U' against the oracle."""
    import torch.multiprocessing as mp
    from tests import native

    native.load()
    out = str(tmp_path / "shard.npz")
    mp.spawn(_gloo_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    r = np.load(out)
    assert int(r["st"]) == 0
    tmap, layers, params, x0, U = _workload(3000, 80, alpha_explore=0.2)
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    S = r["S"].astype(np.float64)
    ks = np.concatenate([np.arange(0, 3000, 97), [1299, 1300, 2999]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 12, ks)
    ok = (np.abs(S[ks] - S_ref) <= REL * np.maximum(np.abs(S_ref), 1.0)) | (margins < 2e-4)
    assert ok.all()
    rc, w_ref, _, _ = oracle.weights(S, P.lam)
    U_ref = oracle.update(P, 12, w_ref, U)
    np.testing.assert_allclose(r["Uo"], U_ref, rtol=0, atol=REL * max(np.abs(U_ref).max(), 0.35))
