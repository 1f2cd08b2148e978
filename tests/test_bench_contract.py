"""Host-side pieces of bench.py: the stored DRAM traffic of the image kernel
is used only while the kernel's source is the captured one and scales with
the showers per launch; the reference arm prints one JSON line with the
fields the measurement contract names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stored_traffic_scales_with_the_launch_and_checks_the_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["supa_voxel_kernel"]["plain30"]
    t = bench.stored_traffic("supa_voxel_kernel", "plain30", rec["showers_per_launch"])
    assert t == rec["bytes_per_launch"]
    assert bench.stored_traffic("supa_voxel_kernel", "plain30", rec["showers_per_launch"] // 8) == pytest.approx(
        rec["bytes_per_launch"] / 8)
    assert bench.stored_traffic("supa_voxel_kernel", "no-such-workload", 1) is None


def test_stored_traffic_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(open(os.path.join(ROOT, "profiles", "traffic.json")).read())
    src = tmp_path / "paper_2202_05012_gb300" / "csrc"
    src.mkdir(parents=True)
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["supa_voxel_kernel"]["plain30"]
    text = open(os.path.join(ROOT, "paper_2202_05012_gb300", "csrc", rec["source"])).read()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (src / rec["source"]).write_text(text)
    assert bench.stored_traffic("supa_voxel_kernel", "plain30", 1) is not None
    (src / rec["source"]).write_text(text + "\n// changed\n")
    assert bench.stored_traffic("supa_voxel_kernel", "plain30", 1) is None


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "plain10",
                          "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"],
                         capture_output=True, text=True, check=True, timeout=600).stdout
    line = json.loads([l for l in out.splitlines() if l.startswith("{")][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
