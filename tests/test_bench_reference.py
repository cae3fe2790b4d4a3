"""bench.py's reference arm (the float64 oracle timed on the host cores) keeps the bench's JSON
contract: one line with impl, metric, value, unit, cpu_baseline and e2e; under torchrun only rank 0
runs and prints, the other ranks exit 0 without work.  CPU only (the oracle runs on the 200 x 200
rank-5 workload)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "plain_fp64_200",
       "--steps", "1", "--warmup", "0"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(CMD, capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_the_bench_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "iters/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("plain_fp64_200")


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_traffic_is_reported_only_for_the_kernel_source_it_was_taken_on(tmp_path, monkeypatch):
    """The DRAM traffic bench.py reports comes from the committed ncu summary of the same kernel
    source (hash of csrc/) and precision; any other source or a missing class gives null."""
    sys.path.insert(0, ROOT)
    import bench
    sha = bench._kernel_source_sha()
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps({"csrc_sha": sha, "classes_fp64": {"orth": 123.0}, "classes_fp32": {"orth": 45.0}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench._traffic_for("orth", "fp64") == 123.0
    assert bench._traffic_for("orth", "fp32") == 45.0
    assert bench._traffic_for("spmm", "fp64") is None
    assert bench._traffic_for("orth", "bf16") is None
    f.write_text(json.dumps({"csrc_sha": "0" * 16, "classes_fp64": {"orth": 123.0}}))
    assert bench._traffic_for("orth", "fp64") is None
