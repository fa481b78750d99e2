"""bench.py on N > 1 ranks: one iteration of N x 2048 samples sharded over the ranks
(itmpc_iterate_shard, an all-gather of the partial records, itmpc_merge_shards).

Two ranks run here on the one GPU of the test machine: the records go through the host
with gloo (ITMPC_BENCH_BACKEND=gloo) since NCCL needs one GPU per rank; no kernel of one
rank waits on another.  Rank 0 must print one JSON line of the benchmark contract."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_bench_sharded_iteration_over_two_ranks():
    env = dict(os.environ, ITMPC_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr",
           "127.0.0.1", "--master-port", str(_port()), "bench.py", "--gpus", "2", "--steps", "5", "--warmup", "3",
           "--no-forms", "--no-cpu-baseline"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    import bench

    assert d["n_gpus"] == 2 and d["scaling"] == "weak" and d["value"] > 0 and d["steps"] == 5
    assert d["config"]["K"] == 2 * bench.K_WORK and d["config"]["K_per_gpu"] == bench.K_WORK
    assert "K-sharded" in d["config"]["parallelism"]
    assert d["gpu_launches"] == 2 * 5
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0
