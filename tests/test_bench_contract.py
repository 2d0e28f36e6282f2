"""The reference arm of bench.py (the CPU oracle) on a small workload, on CPU.

The JSON line must carry the keys the measurement contract names, and under a
multi-rank launch only rank 0 may run and print.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "lowrank500",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return p


def test_reference_arm_prints_the_contract_line():
    p = _run({})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_traffic_is_reported_only_for_unchanged_sources(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from a committed ncu capture only while every source
    file of the measured kernels is byte-identical to the one captured: a changed file
    (here, one byte appended to the second of two) must make it null."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_1704_05528_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "a.cu").write_bytes(b"kernel a\n")
    (csrc / "b.cuh").write_bytes(b"kernel b\n")
    h = hashlib.sha256(b"kernel a\n" + b"kernel b\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"step": {"sources": ["a.cu", "b.cuh"], "source_sha256_16": h, "bytes_per_launch": 1234},
         "old": {"source": "a.cu", "source_sha256_16": hashlib.sha256(b"kernel a\n").hexdigest()[:16],
                 "bytes_per_launch": 99}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("step") == 1234
    assert bench.load_traffic("old") == 99          # a single-source record
    assert bench.load_traffic("missing") is None
    (csrc / "b.cuh").write_bytes(b"kernel b\n ")
    assert bench.load_traffic("step") is None
    assert bench.load_traffic("old") == 99
