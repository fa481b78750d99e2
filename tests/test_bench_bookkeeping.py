"""bench.py's roofline bookkeeping on the host: the DRAM bytes of a committed ncu summary
count only while the summary's source hash matches the kernel source it was taken on, and
every summary the bench reads names the command that made it and runs committed files only."""
import os
import re

import pytest

import bench

PROFILES = os.path.join(bench.ROOT, "profiles")


def _write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_source_hash_follows_content(tmp_path):
    a = _write(tmp_path, "a.cu", "__global__ void k() {}\n")
    b = _write(tmp_path, "b.cu", "__global__ void k() { }\n")
    assert bench.kernel_source_hash([a]) == bench.kernel_source_hash([a])
    assert bench.kernel_source_hash([a]) != bench.kernel_source_hash([b])
    assert bench.kernel_source_hash([a, b]) != bench.kernel_source_hash([b, a])  # order is part of the hash
    assert re.fullmatch(r"[0-9a-f]{12}", bench.kernel_source_hash([a]))


def test_traffic_only_for_the_profiled_source(tmp_path):
    src = _write(tmp_path, "k.cu", "__global__ void k() {}\n")
    h = bench.kernel_source_hash([src])
    good = _write(tmp_path, "good.md", f"# k\n\nkernel_source_sha1: {h}\ntraffic_bytes_per_launch: 4269483\n")
    assert bench.profiled_traffic(good, [src]) == 4269483.0
    stale = _write(tmp_path, "stale.md", "# k\n\nkernel_source_sha1: 0123456789ab\ntraffic_bytes_per_launch: 1\n")
    assert bench.profiled_traffic(stale, [src]) is None
    no_bytes = _write(tmp_path, "nobytes.md", f"# k\n\nkernel_source_sha1: {h}\n")
    assert bench.profiled_traffic(no_bytes, [src]) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md"), [src]) is None
    # a second key in the same summary (the FP8 launch of the tensor-core kernel)
    two = _write(tmp_path, "two.md", f"kernel_source_sha1: {h}\ntraffic_bytes_per_launch: 10\n"
                 "traffic_bytes_per_launch_fp8: 7\n")
    assert bench.profiled_traffic(two, [src]) == 10.0
    assert bench.profiled_traffic(two, [src], key="traffic_bytes_per_launch_fp8") == 7.0
    with open(src, "a") as f:
        f.write("// edited after the capture\n")
    assert bench.profiled_traffic(good, [src]) is None


@pytest.mark.parametrize("name", sorted(bench.FORM_PROFILES))
def test_form_profiles_exist_and_read(name):
    prof, srcs = bench.FORM_PROFILES[name]
    assert os.path.exists(os.path.join(PROFILES, prof)), prof
    for f in srcs:
        assert os.path.exists(os.path.join(bench.ROOT, "paper_1707_02342_gb300", "csrc", f)), f
    v = bench.form_traffic(name)
    assert v is None or v > 0


def _summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith((".md", ".txt")))


@pytest.mark.parametrize("fname", _summaries())
def test_summaries_give_committed_commands(fname):
    """Each summary states the ncu command it came from; the command runs committed files
    only (no working-folder script) and never lets ncu lock the clocks."""
    text = open(os.path.join(PROFILES, fname)).read()
    cmds = [ln for ln in text.splitlines() if re.search(r"\bncu\b", ln) and not ln.lstrip().startswith("|")]
    assert cmds, f"{fname} names no ncu command"
    assert "_work" not in text
    joined = re.sub(r"\\\n\s*", " ", text)  # shell line continuations
    for line in joined.splitlines():
        for cmd in re.findall(r"\bncu (?!-i ).*", line):
            assert "--clock-control none" in cmd, cmd


def test_summaries_stay_small():
    for f in _summaries():
        assert os.path.getsize(os.path.join(PROFILES, f)) < 16384, f
    assert not [f for f in os.listdir(PROFILES) if f.endswith((".ncu-rep", ".nsys-rep", ".qdrep"))]
