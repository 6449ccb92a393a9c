"""The benchmark's reporting plumbing, on the CPU: the reference arm's JSON
line, the roofline arithmetic and the gating of the recorded DRAM traffic
by the kernel sources' hash."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_complete_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "48",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_roofline_arithmetic():
    # 10 launches of 134217728 points in 3.5 ms total: 16 B per point
    r = bench.roofline_of("acoustic_step", (3.5, 10, 134217728.0), 6690.8, "measured", 2.1e9)
    launch_s = 0.35e-3
    assert r["achieved"] == pytest.approx(16 * 134217728 / launch_s / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / 6690.8, abs=1e-4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 2.1e9
    assert r["launches"] == 10 and r["bytes_per_point"] == 16
    r2 = bench.roofline_of("acoustic_step2", (3.5, 10, 134217728.0), 6690.8, "measured")
    assert r2["bytes_per_point"] == 20


def test_recorded_traffic_is_reported_only_for_the_kernel_it_was_measured_on(monkeypatch):
    d = bench.ncu_traffic()
    assert d is not None, "profiles/acoustic_step_traffic.json does not match the kernel sources"
    assert d["kernel_hash"] == bench.kernel_source_hash()
    for so in ("4", "8", "12", "16"):
        # within a few percent of the 16 algorithmic bytes per point
        assert abs(d["acoustic_step"][so] / d["algorithmic_bytes_per_launch"]["acoustic_step"]
                   - 1.0) < 0.05
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic() is None


def test_kernel_hash_ignores_comment_lines_but_not_code(tmp_path, monkeypatch):
    """A whole-line comment edit keeps the hash (the kernel is unchanged); an
    edit of a code line, or of a comment at the end of a code line, changes
    it."""
    import shutil
    src = os.path.join(ROOT, "paper_1807_03032_gb300", "csrc")
    dst = tmp_path / "paper_1807_03032_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("acoustic.cu", "acoustic2.cu", "f32x2.cuh", "common.cuh", "kernels.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    p = dst / "acoustic.cu"
    text = p.read_text()
    p.write_text("// a new whole-line comment\n\n" + text.replace("\n//", "\n    // reworded:", 1))
    assert bench.kernel_source_hash() == h0
    p.write_text(text.replace("int nzc = 1;", "int nzc = 2;", 1))
    assert bench.kernel_source_hash() != h0
    p.write_text(text.replace(";\n", ";  // trailing\n", 1))
    assert bench.kernel_source_hash() != h0
