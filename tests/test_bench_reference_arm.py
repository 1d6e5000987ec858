"""bench.py's reference arm (the CPU oracle timed on a bounded sample of the
3D workload, no GPU) prints one JSON line of the bench contract: the arm's
metric, unit and config, a cpu_baseline describing the run (the OpenMP
cell-parallel build on all host cores, the serial build beside it) and an
e2e record with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("super-droplet-steps/s") and d["unit"] == "SD-steps/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert d["value"] > 0 and cb["value"] == d["value"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["host"]["nproc"] >= 1
    assert cb["serial"]["cores"] == 1 and cb["serial"]["value"] > 0
    # the per-step time is the sample's own, measured by long - short runs
    assert abs(d["ms_per_step"] - cb["ms_per_step"]) < 1e-9
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert "2x2x128 cells" in d["config"]["workload"] and "67108864 SDs" in d["config"]["of"]
