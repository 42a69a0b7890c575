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


def test_traffic_figure_needs_unchanged_sources(tmp_path, monkeypatch):
    """The bench line's `traffic` comes from a stored ncu capture; it is
    reported only while the digest of the sources it depends on is the one
    stored with it, and is null (with the reason) once they change or when no
    capture exists for the kernel and workload."""
    sys.path.insert(0, ROOT)
    import bench

    src = tmp_path / "kernel.cu"
    src.write_text("first version")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", ["kernel.cu"])
    digest = bench.sources_digest(["kernel.cu"])
    monkeypatch.setattr(bench, "TRAFFIC", {("work", "fam"): {"bytes_per_launch": 123.0e6,
                                                             "sources_sha256_16": digest,
                                                             "profile": "profiles/k.md"}})
    value, why = bench.traffic_for("work", "fam")
    assert value == 123.0e6 and "profiles/k.md" in why
    src.write_text("second version")
    value, why = bench.traffic_for("work", "fam")
    assert value is None and "changed" in why
    value, why = bench.traffic_for("work", "other")
    assert value is None and "no ncu capture" in why


def test_stored_traffic_entries_are_well_formed():
    """Every stored capture names an existing profile summary, a 16-hex-digit
    digest and a positive byte count."""
    sys.path.insert(0, ROOT)
    import bench

    for key, t in bench.TRAFFIC.items():
        assert t["bytes_per_launch"] > 0, key
        assert len(t["sources_sha256_16"]) == 16 and int(t["sources_sha256_16"], 16) >= 0, key
        assert os.path.exists(os.path.join(ROOT, t["profile"])), key
    for f in bench.TRAFFIC_SOURCES:
        assert os.path.exists(os.path.join(ROOT, f)), f
