"""The benchmark's reference arm (the CPU oracle on a bounded sample) prints one JSON line
with the keys the benchmark contract names; run on a small box so it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", str(64 ** 3), "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "dtype", "data",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("hacc262144_")


def test_roofline_is_recomputable_from_per_mode_fields():
    # the line's roofline counts the algorithmic bytes of the checks that ran (loss_evals),
    # not of the launches: launches after a stop return at once and move nothing
    sys.path.insert(0, ROOT)
    import bench
    per_mode = {
        "VP": dict(loss_evals=184, pgd_launches=192, n_editable=5_182_479, n_active=43_962_958, ms_pgd_iter=100.0),
        "HF": dict(loss_evals=92, pgd_launches=96, n_editable=3_950_559, n_active=3_409_421, ms_pgd_iter=12.0),
    }
    r = bench.pgd_roofline(per_mode, 6800.0, "measured")
    nbytes = sum((112 * m["n_editable"] + 8 * m["n_active"]) * m["loss_evals"] for m in per_mode.values())
    achieved = nbytes / (112.0 / 1e3) / 1e9
    assert abs(r["achieved"] - achieved) < 0.1
    assert abs(r["frac"] - achieved / 6800.0) < 1e-4
    assert r["checks_per_step"] == 276 and r["launches_per_step"] == 288
    # counting launches instead of checks would overstate the bytes
    wrong = sum((112 * m["n_editable"] + 8 * m["n_active"]) * m["pgd_launches"] for m in per_mode.values())
    assert wrong > nbytes
