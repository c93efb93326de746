"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
runs without a GPU and prints one JSON line in the benchmark's format."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    # the mid workload keeps the CPU suite short; the default (Moana-scale)
    # workload runs the same code on a 261 M-quad scene
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--workload", "mid"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3
    assert d["unit"] == "Mrays/s" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the GPU arm prints the same config dict for the same workload
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.workload_config("mid", 1.0)
    assert set(bench.workload_config("moana", 1.0)) == {"workload", "l2"}


def test_recorded_traffic_needs_current_sources_and_launch_parameters(tmp_path, monkeypatch):
    """A committed DRAM figure is reported only for the kernel sources and the
    launch parameters it was captured with."""
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"moana": {"kernel": "k", "dram_bytes_per_launch": 123, "source": "s",
                     "kernel_source_hash": bench.kernel_source_hash(),
                     "launch": {"block": 256, "fetch": 32, "occupancy": 40}},
           "mid": {"kernel": "k", "dram_bytes_per_launch": 5, "source": "s",
                   "kernel_source_hash": "0000000000000000"}}
    (prof / "roofline_traffic.json").write_text(json.dumps(rec))
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.recorded_traffic("moana")[0] == 123.0          # library defaults
    assert bench.recorded_traffic("moana", {"block": 256, "fetch": 32, "occupancy": 40,
                                            "batch": 1, "stack": 64})[0] == 123.0
    assert bench.recorded_traffic("moana", {"block": 256, "occupancy": 32})[0] is None
    assert bench.recorded_traffic("mid")[0] is None               # other kernel sources
    assert bench.recorded_traffic("tiny")[0] is None
