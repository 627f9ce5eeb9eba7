"""Host-side logic of bench.py (no GPU): the profile fingerprint, the
reference arm's JSON line and the CPU baseline's sample sizing."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_code_ignores_comments_and_blank_space():
    src = "int a = 1; // one\n/* block\n comment */\n\n   int b = 2;\n"
    same = "int a = 1;\n  int b = 2;   // two\n"
    other = "int a = 1;\nint b = 3;\n"
    assert bench.kernel_code(src) == bench.kernel_code(same)
    assert bench.kernel_code(src) != bench.kernel_code(other)


def test_profile_traffic_needs_a_matching_source(tmp_path, monkeypatch):
    """A profile summary is used only while its source fingerprint matches."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "walk_kernel_demo.md").write_text(
        f"x\n\ntraffic_bytes_per_launch: 12345\nkernel_source_sha: {bench.kernel_source_sha()}\n")
    (prof / "walk_kernel_stale.md").write_text(
        "traffic_bytes_per_launch: 999\nkernel_source_sha: 0000000000000000\n")
    real = bench.ROOT
    csrc = os.path.join(real, "paper_2103_02309_gb300")
    os.symlink(csrc, tmp_path / "paper_2103_02309_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("demo") == 12345
    assert bench.profiled_traffic("stale") is None
    assert bench.profiled_traffic("demo", "variant") is None
    assert bench.profiled_traffic("missing") is None


def test_reference_arm_line_on_the_tiny_scene():
    """`--impl reference` times the oracle and prints the contract's line."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baseline_sizes_its_sample_and_times_brute_force():
    import scenegen as sg
    s = sg.make_config("tiny")
    cb = bench.cpu_baseline("tiny", s, dict(bench.WORKLOADS["tiny"]), budget_s=0.5)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert "every 1th pixel" in cb["sample"]          # the whole 64x64 frame fits the budget
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    assert cb["bruteforce"]["value"] > 0 and "192 triangles" in cb["bruteforce"]["sample"]


def test_reference_arm_on_the_batched_workload():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "batched",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC_BATCHED
    assert line["value"] > 0 and line["scaling"] == "strong"
    assert "brute force" in line["cpu_baseline"]["sample"]
