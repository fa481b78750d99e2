"""bench.py's reference arm (the FP64 oracle timed on the host cores) keeps the benchmark
contract on a machine without a GPU: one JSON line from rank 0 with the benchmark's metric,
unit and configuration plus its cpu_baseline and e2e objects; every other rank exits 0
without work or output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line_on_rank_zero():
    r = _run(0, 2)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] >= 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["config"]["K"] == 2 * bench.K_WORK and d["config"]["T"] == bench.T_WORK
    assert d["config"]["K_per_gpu"] == bench.K_WORK  # one iteration of 2 x 2048 samples, as the GPU arm shards it
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(1, 2)
    assert r.returncode == 0 and r.stdout.strip() == ""
