"""bench.py's reference arm on the host (no GPU): it times the FP64 oracle on a
bounded crop of the workload and prints one JSON line with the contract's
keys; under a multi-rank launch only rank 0 works and prints; the timing
rules it enforces (at least 3 warm-up steps) reject a bad command line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    for key in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(key, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_line_has_the_contract_keys():
    p = run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3
    # one step is one oracle pass over a crop (the bounded sample): ms_per_step is
    # that pass's time, and value scales its rate to the whole cube
    assert d["value"] > 0 and d["ms_per_step"] > 0
    frac = 64 * 64 / (256 * 256)
    assert d["value"] == pytest.approx(frac / (d["ms_per_step"] / 1000.0), rel=1e-9)
    assert "crop" in d["config"]["step"]
    assert d["config"]["workload"] == "s3ttv_256x256x128_k5"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] > 0 and cb["value"] == d["value"] and "crop" in cb["sample"]
    assert cb["cpu_model"] and cb["cores_available"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_exit_without_work():
    p = run(["--impl", "reference", "--steps", "1", "--warmup", "3"],
            {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_fewer_than_three_warmup_steps_rejected():
    p = run(["--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=60)
    assert p.returncode != 0 and "warmup" in p.stderr


def test_traffic_figure_follows_the_kernel_sources(monkeypatch):
    """The DRAM traffic bench.py reports comes from an ncu capture of one
    version of the streaming block-dual kernel; it is reported only while
    block_dual.cu and the internal header hash to that capture, and only for
    the block side it was taken at."""
    import bench
    N = 256 * 256 * 128
    sha = bench.block_dual_source_sha()
    assert sha is not None and len(sha) == 16
    monkeypatch.setitem(bench.BLOCK_DUAL_TRAFFIC, "sha", sha)
    got = bench.block_dual_traffic(bench.BLOCK_DUAL_TRAFFIC["k"], N)
    assert got == bench.BLOCK_DUAL_TRAFFIC["bytes_per_voxel"] * N
    assert bench.block_dual_traffic(bench.BLOCK_DUAL_TRAFFIC["k"] + 1, N) is None
    monkeypatch.setitem(bench.BLOCK_DUAL_TRAFFIC, "sha", "0" * 16)
    assert bench.block_dual_traffic(bench.BLOCK_DUAL_TRAFFIC["k"], N) is None
