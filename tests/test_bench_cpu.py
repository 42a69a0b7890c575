"""The benchmark's reference arm (the CPU oracle) prints one JSON line with the
keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["n_gpus"] == 1 and out["steps"] == 1
    assert out["higher_is_better"] is True and out["value"] > 0 and out["unit"] == "steps/s"
    assert abs(out["ms_per_step"] - 1e3 / out["value"]) <= 1e-6 * out["ms_per_step"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert out["config"]["workload"] == "fd2d_n4096"


def test_reference_arm_fits_its_budget(monkeypatch, capsys):
    """With more steps than the wall-time budget allows at the default sample,
    the reference arm shrinks the sample and scales by the O(n^3) cost."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.5)

    class Args:
        workload = "fd2d_n4096"
        steps = 3
        warmup = 2

    bench.run_reference(Args(), 0, 1)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    sample = out["cpu_baseline"]["sample"]
    assert "N=1024" not in sample.split(";")[0] and "by (N/" in sample
    n = int(sample.split("by (N/")[1].split(")")[0])
    assert 256 <= n < 1024 and n % 32 == 0
    assert out["value"] > 0 and out["steps"] == 3
