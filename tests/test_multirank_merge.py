"""Sample-sharded iteration over two ranks (gloo on CPU).

The K samples of one iteration are split into two disjoint shards, one per
rank.  Each rank forms the partial record a GPU shard would produce (rho_s,
eta_s, eta_imp_s, sum e^2, n_finite, E_s) from oracle costs and noise of its
own samples, the records are all-gathered, and the library's host merge
(itmpc_merge_partials, a log-sum-exp merge) must reproduce the unsharded
oracle update.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def shard_record(P, S, ks, it, U, T, stride):
    import oracle

    fin = np.isfinite(S)
    rho = S[fin].min() if fin.any() else np.inf
    e = np.where(fin, np.exp(-(S - rho) / P.lam), 0.0) if np.isfinite(rho) else np.zeros_like(S)
    n_imp = int(np.ceil((1.0 - P.alpha_explore) * P.K))
    rec = np.zeros(stride, np.float64)
    rec[0], rec[1] = rho, e.sum()
    rec[2] = e[ks < n_imp].sum()
    rec[3], rec[4] = (e ** 2).sum(), fin.sum()
    E = np.zeros((T, 2))
    for k, ek in zip(ks, e):
        for t in range(T):
            E[t] += ek * oracle.noise_at(P, it, int(k), t)
    rec[8:8 + 2 * T] = E.reshape(-1)
    return rec.astype(np.float32)


def worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1707_02342_gb300 import inputs, itmpc
    from tests import native, problems

    K, T, it = 96, 12, 4
    P = problems.oracle_problem(problems.params_small(K=K, T=T, alpha_explore=0.25), problems.ellipse_map(),
                                problems.network())
    x0 = problems.x0_for(problems.ellipse_map(), speed=3.0)
    U = inputs.nominal_controls(T, seed=2)
    ks = np.arange(rank * K // world, (rank + 1) * K // world)
    S, _ = oracle.rollout_many(P, x0, U, it, ks)
    stride = itmpc.partial_stride(T)
    rec = torch.tensor(shard_record(P, S, ks, it, U, T, stride))
    recs = [torch.zeros_like(rec) for _ in range(world)]
    dist.all_gather(recs, rec)
    if rank == 0:
        native.load()
        st, U_out = itmpc.merge_partials(torch.stack(recs).numpy(), U, P.lam)
        rc, U_ref, _, _ = oracle.iterate(P, x0, U, it)
        np.save(result_path, np.stack([U_out.astype(np.float64), U_ref]))
        assert st == 0 and rc == 0
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_sharded_merge_matches_unsharded(tmp_path, world):
    from tests import native

    native.load()  # build before spawning
    out = str(tmp_path / "merge.npy")
    mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
    U_out, U_ref = np.load(out)
    np.testing.assert_allclose(U_out, U_ref, rtol=0, atol=1e-6 * max(np.abs(U_ref).max(), 0.35))
