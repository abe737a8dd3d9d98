"""The benchmark's one-line JSON contract for its reference arm: the FP64 oracle timed on the host
cores over a bounded pixel sample, on the same metric and unit as the GPU arm. Runs on the CPU
with a small fixed sample (MLPS_REF_PIXELS)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*args):
    env = dict(os.environ, MLPS_REF_PIXELS="64")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = _reference_line("--steps", "2", "--warmup", "1")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "rays/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["scaling"] == "weak"
    assert d["config"]["sample_pixels_per_step"] == 64 and d["config"]["pass"] == "fwd+bwd"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "64" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_forward_only():
    d = _reference_line("--steps", "1", "--warmup", "0", "--pass", "fwd")
    assert d["config"]["pass"] == "fwd" and d["value"] > 0


def test_traffic_table_entries_expire_with_their_sources(tmp_path, monkeypatch):
    """`roofline.traffic` comes from a committed ncu capture only while every source file the
    entry lists still hashes to the value recorded with it."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    entry = {"kernel": "k", "precision": ["bf16"], "workload": "prec", "bytes_per_launch": 1.5e9,
             "sources": {"k.cu": h}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"mlp_bwd": [entry], "mlp_fwd": []}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("mlp_bwd", "bf16", "prec") == 1.5e9
    assert bench._traffic("mlp_bwd", "fp8", "prec") is None      # no capture for this precision
    assert bench._traffic("mlp_bwd", "bf16", "stress") is None   # nor for this workload
    src.write_text("kernel v2\n")
    assert bench._traffic("mlp_bwd", "bf16", "prec") is None      # the kernel changed since
