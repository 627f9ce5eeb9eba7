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


def test_profile_counters_need_a_matching_source(tmp_path, monkeypatch):
    """A profile summary is used only while its source fingerprint matches."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "walk_kernel_demo.md").write_text(
        f"x\n\ntraffic_bytes_per_launch: 12345\nl2_bytes_per_launch: 67890\n"
        f"kernel_source_sha: {bench.kernel_source_sha()}\n")
    (prof / "walk_kernel_stale.md").write_text(
        "traffic_bytes_per_launch: 999\nkernel_source_sha: 0000000000000000\n")
    real = bench.ROOT
    csrc = os.path.join(real, "paper_2103_02309_gb300")
    os.symlink(csrc, tmp_path / "paper_2103_02309_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_counters("demo") == {"traffic_bytes_per_launch": 12345,
                                               "l2_bytes_per_launch": 67890}
    assert bench.profiled_counters("stale") is None
    assert bench.profiled_counters("demo", "variant") is None
    assert bench.profiled_counters("missing") is None


def test_walk_roofline_counts_the_methods_bytes():
    """The walk's fraction counts 32 B per tet step (Tet16 record + float4
    point) whatever record the walk reads; the record's own bytes, the
    per-ray bytes over the trace and the ncu DRAM / L2 fractions sit beside it."""
    steps, rays = 1_000_000_000, 10_000_000
    prof = {"traffic_bytes_per_launch": 1e9, "l2_bytes_per_launch": 4e9}
    r = bench.walk_roofline(steps, rays, walk_ms=4.0, trace_ms=5.0, step_ms=6.0, hbm=8000.0,
                            hbm_src="measured", l2_peak=6000.0, record_bytes=16, prof=prof,
                            kind="bounce")
    assert r["bytes_per_tet_step"] == 32 and r["bytes_per_ray"] == 188
    assert r["achieved"] == 8000.0 and r["frac"] == 1.0            # 32 GB in 4 ms
    assert r["frac_record_bytes"] == 0.5
    assert r["frac_trace"] == round((32e9 + 188 * rays) / 5e-3 / 1e9 / 8000.0, 4)
    assert r["dram_frac"] == 0.0625                                # 1 GB per 2 ms launch
    assert r["l2_frac"] == round(4e9 / 2e-3 / 1e9 / 6000.0, 4)
    assert r["dram_over_algorithmic"] == round(1e9 / 16e9, 4)       # 16 GB a launch
    assert r["l2_over_algorithmic"] == 0.25
    assert r["tflops"] == round(13e9 / 4e-3 / 1e12, 2)
    none = bench.walk_roofline(steps, rays, 4.0, 5.0, 6.0, 8000.0, "measured", 6000.0, 16, None,
                               "bounce")
    assert none["traffic"] is None and none["dram_frac"] is None and none["l2_frac"] is None


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
    assert "every pixel" in cb["sample"]              # the whole 64x64 frame fits the budget
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


def test_oracle_leg_compares_every_ray_of_every_arm():
    """The bench's oracle leg on the tiny scene, with frames made from the
    oracle's own hits (packed as the device writes them): every arm meets the
    parity bar; one planted wrong triangle in one arm is an unexcused
    mismatch there and nowhere else."""
    import numpy as np
    import oracle
    import scenegen as sg
    from oracle.secondary import hit_side, secondary_rays
    from paper_2103_02309_gb300 import tetmesh as tmx
    s = sg.make_config("tiny")
    W = dict(bench.WORKLOADS["tiny"])
    om = oracle.OracleMesh(s.points, s.tets, s.tris)
    cam, _ = om.locate(np.array([s.camera.eye], np.float32))
    o, d = sg.camera_rays(s.camera)
    w = om.trace(o, d, np.inf, cam[0])

    def pack(r):
        h = np.zeros((len(r["tri"]), 8), np.int32)
        f = h.view(np.float32)
        h[:, 0] = r["tri"]
        f[:, 1], f[:, 2], f[:, 3] = r["t"], r["b1"], r["b2"]
        return h
    side = hit_side(om.arrays()[2], w["tri"], w["tet"])
    o2, d2, tm2, entry, _ = secondary_rays(s.points, s.tris, w["tri"], np.float32(w["b1"]),
                                           np.float32(w["b2"]), side, 5, 1, np.inf)
    rays2 = tmx.pack_rays(o2, d2, tm2, -1 - entry)
    w2 = om.trace(o2, d2, tm2, -1, entry)
    good = dict(hits=pack(w), rays2=rays2, hits2=pack(w2))
    bad = {k: v.copy() for k, v in good.items()}
    far = int(np.nonzero(w2["tri"] >= 0)[0][0])
    bad["hits2"][far, 0] = (w2["tri"][far] + 17) % s.n_tris     # a hit on another triangle
    cpu, vs = bench.oracle_leg("tiny", s, W, {"fp32g": good, "fp64": bad}, tmx, budget_s=0.3)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0
    a = vs["fp32g"]
    assert a["meets_bar"] and a["primary"]["agree"] == 1.0 and a["secondary"]["agree"] == 1.0
    assert a["primary"]["n"] == s.camera.width * s.camera.height
    assert a["secondary"]["n"] == len(o2)
    b = vs["fp64"]
    assert not b["meets_bar"] and b["secondary"]["unexcused"] == 1 and b["primary"]["mismatches"] == 0
    assert "every ray" in vs["sample"]


def test_committed_walk_profiles_carry_their_counters_and_source():
    """The ncu summaries that the bench's rooflines quote (the default walk
    and the Tet16 arm's walk on the precision workload) hold DRAM and L2
    bytes per launch and the hash of the kernel source they were taken
    from; the bench uses them only while that hash is current."""
    import re
    for name in ("precision", "precision_tet16"):
        text = open(os.path.join(bench.ROOT, "profiles", f"walk_kernel_{name}.md")).read()
        for key in ("traffic_bytes_per_launch", "l2_bytes_per_launch"):
            m = re.search(rf"^{key}: *(\d+)", text, re.M)
            assert m and int(m.group(1)) > 0, (name, key)
        assert re.search(r"^kernel_source_sha: *[0-9a-f]{16}$", text, re.M), name
        got = bench.profiled_counters(name)
        assert got is None or got["traffic_bytes_per_launch"] > 0
