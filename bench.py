#!/usr/bin/env python3
"""Throughput of constrained tet-mesh ray traversal on one GB300 (or N replicas).

Workload (default, "precision"): 128^3-cell Kuhn grid over [0,1]^3
(12,582,912 tets, 2,146,689 points, jitter +-0.15 cell), constrained surface
of 64 seeded random spheres, pinhole camera at (0.5, 0.5, 0.02) looking +z
with a 70 degree field of view, 2048x2048 primary rays plus one
cosine-weighted diffuse bounce per hit.  One step = locate the camera tet,
generate the primary rays, trace them, generate the bounce rays from the
hits, trace those (all on the device).  Metric: Mrays/s (primary + bounce)
with the FP32 walk and FP64 guard; the all-FP64 and pure-FP32 arms run the
same step on the same inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other measurements on the same step (each prints its own JSON line):
  --workload medium|large|tiny|batched   other scene sizes (large: 8 AO rays per hit)
  --order hilbert|input|hilbert_regions  memory order of the mesh (Sec. 5)
  --format tet16|tet20|tet20_aos|tet32|face|face16
                                         record the walk reads: the paper's (Sec. 3)
                                         or face entries (default: 16-byte ones)
  --secondary bounce|ao|shadow|reflect|refract
                                         the rays generated from the primary hits
                                         (Sec. 6; shadow rays go to a point light
                                         located on the device every step)

The line also carries the walk's roofline (algorithmic bytes over its event
time against the measured HBM copy rate, beside the L2 read rate the library's
probe measures here), `e2e` (host rays in, host hits out, copies inside the
timed region, two slices through a copy-in / trace / copy-out pipeline), the
CPU oracle's rate on a bounded sample, and the SM clocks seen while timing.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mrays/s (primary + diffuse-bounce) at 1 GB300 vs all-FP64 GPU path; %BW roofline"
UNIT = "Mrays/s"
METRIC_BATCHED = "Mrays/s, 32-mesh uneven batch in one persistent graph launch"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
RAY_BYTES, HIT_BYTES = 32, 32
# Algorithmic bytes of the walk kernel (the dominant kernel): per tet step one
# tet record (RECORD_BYTES of the format the walk reads) and one float4
# point; per ray its start record (32 B, in the hit slot), the ray (32 B),
# the three entry-face points (48 B) and the end record (32 B).
# The method's algorithmic bytes (the paper's compact layout, whatever record
# the walk reads): per tet step the 16-byte Tet16 record and the 16-byte
# float4 point of the new vertex; per ray its 36-byte ray, 32-byte hit, the
# start tet's 32-byte full record and four 16-byte points, and the 24-byte
# triangle record of the hit.
METHOD_STEP_BYTES = 16 + 16
METHOD_RAY_BYTES = 36 + 32 + 32 + 4 * 16 + 24
# What the walk kernel of each record format reads per step (record + point).
RECORD_BYTES = {"tet16": 16, "tet20": 20, "tet20_aos": 20, "tet32": 32, "face": 32, "face16": 16}
POINT_BYTES = {"face": 0, "face16": 0}   # face entries carry the new vertex; the others read a point
MODE_NAMES = {"fp32g": "FP32 walk + FP64 guard", "fp32": "pure FP32", "fp64": "all FP64"}
# Rays generated from each hit: (rays per hit, tmax); None = per-ray (shadow)
SECONDARY = {"bounce": (1, float("inf")), "ao": (8, 0.05), "shadow": (1, None),
             "reflect": (1, float("inf")), "refract": (1, float("inf"))}
LIGHT = (0.3, 0.75, 0.05)   # point light of the shadow measurement (inside the unit cube)
IOR = 1.5                   # refractive index of the inside of the spheres
E2E_CHUNKS = int(os.environ.get("TM_E2E_CHUNKS", "2"))    # e2e: frame slices
E2E_STREAMS = int(os.environ.get("TM_E2E_STREAMS", "2"))  # e2e: streams they go round

WORKLOADS = {
    "tiny": dict(desc="8^3-cell Kuhn grid (3,072 tets), one sphere, 64x64 primary rays + 1 cosine "
                      "bounce per hit", per_hit=1, tmax=float("inf"), kind="bounce"),
    "precision": dict(desc="128^3-cell Kuhn grid (12,582,912 tets, 2,146,689 points, jitter 0.15), "
                           "64 random spheres, 2048x2048 primary rays + 1 cosine bounce per hit",
                      per_hit=1, tmax=float("inf"), kind="bounce", format="face16"),
    "medium": dict(desc="64^3-cell Kuhn grid (1,572,864 tets), 16 random spheres, 1920x1080 "
                        "primary rays + 1 cosine bounce per hit",
                   per_hit=1, tmax=float("inf"), kind="bounce"),
    "large": dict(desc="256^3-cell Kuhn grid (100,663,296 tets), 256 random spheres, 1024x1024 "
                       "primary rays + 8 ambient-occlusion rays per hit (t_max 0.05)",
                  per_hit=8, tmax=0.05, kind="ao", format="face16"),
    "batched": dict(desc="32 meshes of 16^3..96^3 cells with 4-32 random spheres each, 1K-2M rays "
                         "per mesh (log-uniform), half camera rays and half uniform-direction rays "
                         "from located interior points", per_hit=0, tmax=float("inf"), kind="none"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="precision")
    p.add_argument("--order", choices=["hilbert", "input", "hilbert_regions"], default="hilbert")
    p.add_argument("--format", choices=sorted(RECORD_BYTES), default=None,
                   help="tet record the walk reads (default: 16-byte face entries, the "
                        "library's automatic choice when built)")
    p.add_argument("--secondary", choices=sorted(SECONDARY), default=None,
                   help="rays generated from the primary hits (default: the workload's)")
    p.add_argument("--split", choices=["replicas", "tiles"], default="replicas",
                   help="with N ranks: every rank traces a whole frame of its own (replicas, "
                        "weak scaling), or the ranks split one frame by pixel tiles and gather "
                        "its hits to rank 0 inside the timed step (tiles, strong scaling)")
    p.add_argument("--cells", type=int, default=0,
                   help="grid cells per axis instead of the workload's (a reduced case of the "
                        "same scene recipe, e.g. for counter captures)")
    p.add_argument("--eager", action="store_true",
                   help="time the step as separate API calls instead of replaying it from a "
                        "CUDA graph captured from the same calls")
    p.add_argument("--no-arms", action="store_true", help="skip the FP64 / FP32 comparison arms")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--refill", type=int, default=0)
    p.add_argument("--batch-steps", type=int, default=0)
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def read_probe(torch, buf, reps, sink):
    """The benchmark's read-bandwidth probe (libtmprobe.so, built beside the
    library and kept out of its C ABI): `reps` passes over `buf`."""
    import ctypes
    from paper_2103_02309_gb300 import build as libbuild
    lib = ctypes.CDLL(libbuild.PROBE_LIB)
    fn = lib.tm_bench_read_probe
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    st = fn(buf.data_ptr(), buf.numel() * buf.element_size(), int(reps), sink.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise RuntimeError(f"tm_bench_read_probe failed with status {st}")


def measured_l2(torch, tmx, dev, mib=48, reps=40):
    """Read bandwidth of a buffer resident in L2 (GB/s): the L2 roofline of
    workloads whose records fit in L2.  The read probe over `mib` MiB, first
    passes untimed so the buffer is resident, then `reps` timed."""
    x = torch.ones(mib * (1 << 20) // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    read_probe(torch, x, 3, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    read_probe(torch, x, reps, sink)
    e1.record()
    e1.synchronize()
    return x.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
            return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_code(text):
    """Source text without comments and blank space, so that a comment edit
    does not mark a profile of the same code as stale."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.strip() for line in text.splitlines() if line.strip())


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("trace.cu", "walk.cuh"):  # the walk kernel's sources
        with open(os.path.join(ROOT, "paper_2103_02309_gb300", "csrc", f)) as fh:
            h.update(kernel_code(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_counters(workload, variant=""):
    """ncu counters per walk launch from the committed summary
    (profiles/walk_kernel_<workload>.md): DRAM bytes (`traffic_bytes_per_launch`)
    and L2 bytes (`l2_bytes_per_launch`), or None when the summary was taken
    from other kernel source than the current one, or for a variant run."""
    if variant:
        return None
    path = os.path.join(ROOT, "profiles", f"walk_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    keys = ("traffic_bytes_per_launch", "l2_bytes_per_launch", "kernel_source_sha")
    for line in open(path):
        if ":" in line and line.strip().startswith(keys):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha") != kernel_source_sha():
        return None
    out = {}
    for k in ("traffic_bytes_per_launch", "l2_bytes_per_launch"):
        try:
            out[k] = float(vals[k])
        except (KeyError, ValueError):
            out[k] = None
    return out


def walk_roofline(tet_steps, rays, walk_ms, trace_ms, step_ms, hbm, hbm_src, l2_peak,
                  record_bytes, prof, kind):
    """The walk kernel's roofline for one step (two walk launches: primary
    and secondary rays).  `frac` counts the method's algorithmic bytes (the
    Tet16 record and the float4 point per tet step) over the walk's event
    time against the measured HBM copy rate; `frac_trace` adds the per-ray
    bytes over the whole trace (start, walk, finish).  The bytes the walk
    fetches from DRAM and moves through L2 per launch (ncu, when the
    committed summary matches this source) give `dram_frac` and `l2_frac`."""
    alg = tet_steps * METHOD_STEP_BYTES
    achieved = alg / (walk_ms * 1e-3) / 1e9
    trace_alg = alg + rays * METHOD_RAY_BYTES
    rec = tet_steps * record_bytes
    walk_s_launch = walk_ms * 1e-3 / 2
    traffic = prof.get("traffic_bytes_per_launch") if prof else None
    l2b = prof.get("l2_bytes_per_launch") if prof else None
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic,
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured"
            else "fallback 6.8 TB/s",
            "kernel": f"walk_kernel (primary + {kind} launches; bytes and time per step)",
            "bytes_per_tet_step": METHOD_STEP_BYTES,
            "bytes_per_ray": METHOD_RAY_BYTES,
            "algorithmic_bytes_per_launch": alg // 2,
            "walk_ms_per_launch": round(walk_ms / 2, 4),
            "tet_steps_per_step": tet_steps,
            "frac_trace": round(trace_alg / (trace_ms * 1e-3) / 1e9 / hbm, 4),
            "record_bytes_per_tet_step": record_bytes,
            "frac_record_bytes": round(rec / (walk_ms * 1e-3) / 1e9 / hbm, 4),
            "dram_frac": round(traffic / walk_s_launch / 1e9 / hbm, 4) if traffic else None,
            "l2_bytes": l2b,
            "l2_frac": round(l2b / walk_s_launch / 1e9 / l2_peak, 4) if l2b else None,
            # what the hardware moved against the method's bytes (per launch)
            "dram_over_algorithmic": round(traffic / (alg / 2), 4) if traffic else None,
            "l2_over_algorithmic": round(l2b / (alg / 2), 4) if l2b else None,
            # the paper's count of about 13 FP32 operations per tet step,
            # over the walk time: reported, not the bound
            "flops_per_tet_step": 13,
            "tflops": round(tet_steps * 13 / (walk_ms * 1e-3) / 1e12, 2),
            "l2_read_peak_gbs": round(l2_peak, 1),
            "l2_peak_source": "measured here: a read probe (L1-bypassing 16-byte loads) over a "
                              "48 MiB buffer resident in L2",
            "walk_share_of_step": round(walk_ms / step_ms, 4),
            "trace_share_of_step": round(trace_ms / step_ms, 4)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_scene(workload, cells=0):
    import scenegen as sg
    return sg.make_config(workload, n_override=cells or None)


# --------------------------------------------------------------------------- #
# GPU arm


def run_ours(args, world, rank, local):
    import torch
    from paper_2103_02309_gb300 import build as libbuild
    if rank == 0 or not os.path.exists(libbuild.LIB):
        libbuild.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2103_02309_gb300 import tetmesh as tmx
    from paper_2103_02309_gb300.shard import gather_rows, max_over_ranks, shard_seed, tile_range

    W = dict(WORKLOADS[args.workload])
    if args.format is None:
        args.format = W.get("format", "face16")
    kind = args.secondary or W["kind"]
    if kind != W["kind"]:
        W["per_hit"], W["tmax"] = SECONDARY[kind]
        W["kind"] = kind
    s = build_scene(args.workload, args.cells)
    t0 = time.time()
    mesh = tmx.Mesh(s.points, s.tets, s.tris, order=args.order,
                    tet20=args.format.startswith("tet20"), faces=args.format == "face",
                    faces16=args.format == "face16")
    build_s = time.time() - t0
    cam = tmx.make_camera(s.camera.eye, s.camera.fov_deg, s.camera.width, s.camera.height)
    n_primary = s.camera.width * s.camera.height
    per_hit = W["per_hit"]
    default_run = (kind == WORKLOADS[args.workload]["kind"]
                   and args.format == WORKLOADS[args.workload].get("format", "face16")
                   and args.order == "hilbert" and not args.cells)
    # one frame split by pixel tiles: this rank's rays [lo, hi), and the seed
    # that gives its secondary rays the whole frame's random draws
    tiles = args.split == "tiles"
    lo, hi = tile_range(n_primary, world, rank) if tiles else (0, n_primary)
    seed2 = shard_seed(0x5EED, lo, per_hit) if tiles else 0x5EED
    dev = torch.device("cuda", local)
    eye = torch.tensor([s.camera.eye], dtype=torch.float32, device=dev)
    start = torch.empty(1, dtype=torch.int32, device=dev)
    rays = torch.empty((n_primary, 8), dtype=torch.float32, device=dev)
    hits = torch.empty((n_primary, 8), dtype=torch.int32, device=dev)
    rays2 = torch.empty((n_primary * per_hit, 8), dtype=torch.float32, device=dev)
    hits2 = torch.empty((n_primary * per_hit, 8), dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)
    light = torch.tensor([LIGHT], dtype=torch.float32, device=dev)
    light_tet = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    ev_p = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev_p + ev_b:
        e.record(stream)                                  # materialise the CUDA events
    torch.cuda.synchronize()

    def opts(mode, ev=None, secondary=False, fmt=None):  # ev=None: no phase events (graph capture)
        # early exit at t_max for the secondary rays with a finite t_max only
        # (primary rays are unbounded)
        bounded = secondary and W["tmax"] is not None and math.isfinite(W["tmax"])
        return tmx.trace_opts(mode=mode, block=args.block, refill=args.refill,
                              batch_steps=args.batch_steps, tmax_early_exit=bounded,
                              phase_events=ev, format=fmt or args.format)

    r1, h1 = rays[lo:hi], hits[lo:hi]                     # the whole frame unless split by tiles

    def step(op, ob):
        mesh.locate(eye, out=start)
        if kind == "shadow":
            mesh.locate(light, out=light_tet)          # the point light, once per frame
        tmx.gen_primary(cam, start, rays=rays)
        mesh.trace(r1, hits=h1, opts=op)
        if kind in ("bounce", "ao"):
            mesh.gen_secondary(h1, per_hit, W["tmax"], seed=seed2, rays_out=rays2, count=count)
            mesh.trace(rays2, hits=hits2, n_dev=count, opts=ob)
        elif kind == "shadow":
            mesh.gen_shadow(h1, LIGHT, rays_out=rays2, count=count)
            mesh.trace_shadow(rays2, light_tet, hits=hits2, n_dev=count, opts=ob)
        else:
            mesh.gen_specular(r1, h1, kind, IOR, rays_out=rays2, count=count)
            mesh.trace(rays2, hits=hits2, n_dev=count, opts=ob)
        if tiles and world > 1:
            # rank 0 collects the frame's hits in pixel-tile order
            gather_rows(h1, world, rank, device=dev)
            gather_rows(hits2[: int(count.item())], world, rank, device=dev)

    # A step replays from a CUDA graph captured from the same API calls
    # (one launch of the whole step instead of about thirty host calls),
    # except for the tile split across ranks, whose gather synchronises with
    # the host.  Phase times come from eager steps with the phase events.
    use_graph = not args.eager and not (tiles and world > 1)

    def timed(mode, steps, warmup, fmt=None):
        op, ob = opts(mode, ev_p, fmt=fmt), opts(mode, ev_b, secondary=True, fmt=fmt)
        for _ in range(warmup):
            step(op, ob)
        torch.cuda.synchronize()
        # phase times (start, walk, finish of both launches) from eager steps
        n_phase = min(steps, 5)
        phases = np.zeros((2, 3))                           # [primary, secondary] x [start, walk, finish]
        trace_ms = walk_ms = 0.0
        per_step = 0
        for _ in range(n_phase):
            flush.zero_()
            l0 = tmx.launch_count()
            step(op, ob)
            torch.cuda.synchronize()
            per_step = tmx.launch_count() - l0
            trace_ms += ev_p[0].elapsed_time(ev_p[3]) + ev_b[0].elapsed_time(ev_b[3])
            walk_ms += ev_p[1].elapsed_time(ev_p[2]) + ev_b[1].elapsed_time(ev_b[2])
            for i, ev in enumerate((ev_p, ev_b)):
                for j in range(3):
                    phases[i, j] += ev[j].elapsed_time(ev[j + 1])
        timed.phases = (phases / n_phase).round(4).tolist()
        run = lambda: step(op, ob)  # noqa: E731
        if use_graph:
            g = torch.cuda.CUDAGraph()
            opg, obg = opts(mode, fmt=fmt), opts(mode, secondary=True, fmt=fmt)
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                step(opg, obg)
            stream.wait_stream(side)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                step(opg, obg)
            g.replay()
            torch.cuda.synchronize()
            run = g.replay
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = tmx.launch_count()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()                                  # evict the mesh from L2 between steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        launches = per_step * steps if use_graph else tmx.launch_count() - l0
        if world > 1:
            torch.distributed.barrier()
        tot = max_over_ranks(tot, dev)                     # the slowest replica's time
        return tot / steps, trace_ms / n_phase, walk_ms / n_phase, launches

    def capture():
        """Host copies of the frame the last step traced: primary hits, the
        rays generated from them, and their hits."""
        k = int(count.item())
        return dict(hits=hits.cpu().numpy(), rays2=rays2[:k].cpu().numpy(),
                    hits2=hits2[:k].cpu().numpy())

    # headline arm: FP32 walk with FP64 guard
    with ClockSampler(local) as clk:
        ms, trace_ms, walk_ms, launches = timed("fp32g", args.steps, max(args.warmup, 3))
    frames = {"fp32g": capture()}
    phase_ms = {"primary": dict(zip(("start", "walk", "finish"), timed.phases[0])),
                "secondary": dict(zip(("start", "walk", "finish"), timed.phases[1])),
                "note": "event-timed per launch, eager steps (start: basis and first tet; finish: the hit)"}
    n_second = int(count.item())
    if tiles and world > 1:
        import torch.distributed as dist
        tot = torch.tensor([n_second], dtype=torch.int64, device=dev)
        dist.all_reduce(tot)
        rays_per_step = n_primary + int(tot.item())   # the frame's rays, over all ranks
    else:
        rays_per_step = n_primary + n_second
    g1 = tmx.unpack_hits(hits)
    g2 = tmx.unpack_hits(hits2[:n_second])
    steps_total = int(g1["steps"].astype(np.int64).sum() + g2["steps"].astype(np.int64).sum())
    record_bytes = RECORD_BYTES[args.format] + POINT_BYTES.get(args.format, 16)
    value = (1 if tiles else world) * rays_per_step / (ms * 1e-3) / 1e6
    extra = {}
    if kind == "shadow":
        extra = {"light": LIGHT, "light_tet": int(light_tet.item()),
                 "lit_rate": float(((g2["flags"] & tmx.HIT_REACHED) != 0).mean()) if n_second else 0.0}
    elif kind in ("reflect", "refract"):
        extra = {"ior": IOR, "secondary_hit_rate": float((g2["tri"] >= 0).mean()) if n_second else 0.0}

    hbm, hbm_src = measured_hbm()
    l2_peak = measured_l2(torch, tmx, dev)
    prof = profiled_counters(args.workload, "" if default_run else "variant")
    roofline = walk_roofline(steps_total, rays_per_step, walk_ms, trace_ms, ms, hbm, hbm_src,
                             l2_peak, record_bytes, prof, kind)

    arms = {}
    if not args.no_arms:
        keep = (hits.clone(), hits2.clone(), rays2.clone(), count.clone())
        arm_list = [("fp64", args.format), ("fp32", args.format)]
        if args.format != "tet16":
            arm_list.append(("fp32g", "tet16"))   # the paper's compact record, same step
        for mode, fmt in arm_list:
            name = mode if fmt == args.format else fmt
            ams, atr, awk, _ = timed(mode, max(2, args.steps // 3), 1, fmt=fmt)
            frames[name] = capture()
            k = int(count.item())
            arms[name] = {"value": round(world * (n_primary + k) / (ams * 1e-3) / 1e6, 2),
                          "ms_per_step": round(ams, 3), "trace_ms": round(atr, 3),
                          "walk_ms": round(awk, 3), "mode": MODE_NAMES[mode], "format": fmt}
            if fmt == "tet16":
                a1, a2 = tmx.unpack_hits(hits), tmx.unpack_hits(hits2[:k])
                st = int(a1["steps"].astype(np.int64).sum() + a2["steps"].astype(np.int64).sum())
                arms[name]["roofline"] = walk_roofline(st, n_primary + k, awk, atr, ams, hbm, hbm_src,
                                                       l2_peak, RECORD_BYTES["tet16"] + 16,
                                                       profiled_counters(
                                                           f"{args.workload}_tet16",
                                                           "" if default_run else "variant"),
                                                       kind)
        arms["fp32g_speedup_vs_fp64"] = round(value / arms["fp64"]["value"], 2)
        hits.copy_(keep[0]); hits2.copy_(keep[1]); rays2.copy_(keep[2]); count.copy_(keep[3])

    info = mesh.info
    nt = s.n_tets
    face_bytes = {"face16": 64, "face": 128}.get(args.format, 0) * nt
    memory = {"device_bytes": int(info.device_bytes),
              "device_bytes_per_tet": round(info.device_bytes / nt, 2),
              "walk_record_bytes_per_tet": {"tet16": 16, "tet20": 20, "tet20_aos": 20, "tet32": 32,
                                            "face": 128, "face16": 64}[args.format],
              "device_bytes_per_tet_without_face_entries": round((info.device_bytes - face_bytes) / nt, 2),
              "note": "per tet: 16 B Tet16 + 32 B cold record (start phase) + face entries when "
                      "the walk reads them; points, triangle and restart records spread over the tets"}

    e2e = None
    if not args.no_e2e and kind in ("bounce", "ao"):
        e2e = run_e2e(args, mesh, tmx, torch, s, cam, n_primary, per_hit, W, dev, world,
                      fmt=args.format)

    cpu = None
    vs_oracle = None
    if not args.no_cpu and world == 1 and rank == 0 and kind in ("bounce", "ao"):
        cpu, vs_oracle = oracle_leg(args.workload, s, W, frames, tmx, budget_s=20.0)

    if rank == 0:
        fl1, fl2 = g1["flags"], g2["flags"]
        fl = np.concatenate([fl1, fl2])

        def rate(a, bit):
            return float(((a & bit) != 0).mean()) if len(a) else 0.0
        metric = METRIC if kind == WORKLOADS[args.workload]["kind"] else f"Mrays/s (primary + {kind})"
        line = {
            "metric": metric, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "strong" if tiles else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {W['desc']}"
                       + (f" (reduced to {args.cells}^3 cells)" if args.cells else ""),
                       "mode": "FP32 walk + FP64 guard",
                       "tets": s.n_tets, "points": s.n_points, "triangles": s.n_tris,
                       "rays_per_step": rays_per_step, "primary": n_primary, "secondary": n_second,
                       "order": args.order, "format": args.format, "secondary_kind": kind,
                       "parallelism": (f"one frame split by pixel tiles over {world} ranks, "
                                       "hits gathered to rank 0" if tiles and world > 1
                                       else f"replicas x{world}" if world > 1 else "1 GPU"),
                       "rays_this_rank": [lo, hi],
                       "l2": "flushed between steps (256 MiB write outside the step events)",
                       "launch": ("each step replayed from a CUDA graph captured from the API calls; "
                                  "phase times from eager steps") if use_graph else
                                 "each step as separate API calls",
                       "build_s": round(build_s, 2), **extra},
            # how often each double-precision path ran (fraction of the step's rays)
            "fp64_paths": {"guard_rate_primary": rate(fl1, tmx.HIT_GUARD),
                           "guard_rate_all": rate(fl, tmx.HIT_GUARD),
                           "final_fp64_rate": rate(fl, tmx.HIT_FINAL_FP64),
                           "restart_3d_rate": rate(fl2, tmx.HIT_RESTART_3D),
                           "start_moved_rate": rate(fl, tmx.HIT_START_MOVED),
                           "parked_rate": rate(fl, tmx.HIT_SLOW_PASS),
                           "tie_rate": rate(fl, tmx.HIT_TIE),
                           "bad_start_rate": rate(fl, tmx.HIT_BAD_START)},
            "roofline": roofline, "phase_ms": phase_ms, "arms": arms, "memory": memory,
            "vs_oracle": vs_oracle,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(args, mesh, tmx, torch, s, cam, n_primary, per_hit, W, dev, world, fmt="auto"):
    """Host rays in, host hits out, through the public API, copies inside the timed region.

    A three-stage pipeline over the frame cut into `E2E_CHUNKS` slices: one
    stream copies the slices' rays in, `E2E_STREAMS` streams trace them
    (primary rays, secondary generation, secondary rays), one stream copies
    the hits out (a slice's primary hits as soon as their trace ends).  Events
    order the stages of each slice, so one step's copies overlap the walks of
    the step before and after it.  The timed region spans all steps, and every
    step copies its whole input in and all its hits out.
    """
    from paper_2103_02309_gb300.shard import shard_seed
    start = mesh.locate(torch.tensor([s.camera.eye], dtype=torch.float32, device=dev))
    rays_dev = tmx.gen_primary(cam, start)
    rays_host = torch.empty_like(rays_dev, device="cpu").pin_memory()
    rays_host.copy_(rays_dev)
    K = max(1, min(E2E_CHUNKS, n_primary))
    bounds = [n_primary * c // K for c in range(K + 1)]
    cin, cout = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    comp = [torch.cuda.Stream(device=dev) for _ in range(max(1, E2E_STREAMS))]
    chunks = []
    for c in range(K):
        m = bounds[c + 1] - bounds[c]
        chunks.append(dict(
            lo=bounds[c], hi=bounds[c + 1],
            rays=torch.empty((m, 8), dtype=torch.float32, device=dev),
            hits=torch.empty((m, 8), dtype=torch.int32, device=dev),
            rays2=torch.empty((m * per_hit, 8), dtype=torch.float32, device=dev),
            hits2=torch.empty((m * per_hit, 8), dtype=torch.int32, device=dev),
            count=torch.empty(1, dtype=torch.int64, device=dev),
            hits_host=torch.empty((m, 8), dtype=torch.int32).pin_memory(),
            hits2_host=torch.empty((m * per_hit, 8), dtype=torch.int32).pin_memory(),
            count_host=torch.empty(1, dtype=torch.int64).pin_memory(),
            in_ready=torch.cuda.Event(), prim_done=torch.cuda.Event(),
            comp_done=torch.cuda.Event(), out_done=torch.cuda.Event()))
    o = tmx.trace_opts(mode="fp32g", format=fmt)
    o2 = tmx.trace_opts(mode="fp32g", tmax_early_exit=math.isfinite(W["tmax"]), format=fmt)
    main = torch.cuda.current_stream(dev)

    def step():
        for c, ch in enumerate(chunks):
            st = comp[c % len(comp)]
            cin.wait_event(ch["prim_done"])     # the previous step's primary trace read the slice
            with torch.cuda.stream(cin):
                ch["rays"].copy_(rays_host[ch["lo"]:ch["hi"]], non_blocking=True)
            ch["in_ready"].record(cin)
            st.wait_event(ch["in_ready"])
            st.wait_event(ch["out_done"])       # the previous step's hits of the slice are home
            mesh.trace(ch["rays"], hits=ch["hits"], opts=o, stream=st)
            ch["prim_done"].record(st)
            # the slice's rays draw the whole frame's random numbers
            mesh.gen_secondary(ch["hits"], per_hit, W["tmax"], seed=shard_seed(0x5EED, ch["lo"], per_hit),
                               rays_out=ch["rays2"], count=ch["count"], stream=st)
            mesh.trace(ch["rays2"], hits=ch["hits2"], n_dev=ch["count"], opts=o2, stream=st)
            ch["comp_done"].record(st)
            cout.wait_event(ch["prim_done"])
            with torch.cuda.stream(cout):
                ch["hits_host"].copy_(ch["hits"], non_blocking=True)
            cout.wait_event(ch["comp_done"])
            with torch.cuda.stream(cout):
                ch["hits2_host"].copy_(ch["hits2"], non_blocking=True)
                ch["count_host"].copy_(ch["count"], non_blocking=True)
            ch["out_done"].record(cout)

    def run(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for st in [cin, cout] + comp:
            st.wait_event(e0)
        for _ in range(n):
            step()
        for st in [cin, cout] + comp:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)
        e1.record(main)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def graph_of(n):
        """The pipeline's n steps captured into one CUDA graph from the same
        API calls: the copy and compute streams fork from the capture
        stream and join it again, and every event a step waits on is first
        recorded inside the capture."""
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(main)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cap):
            for st in [cin, cout] + comp:
                st.wait_stream(cap)
            for ch in chunks:
                for k in ("prim_done", "out_done"):
                    ch[k].record(cap)
            for _ in range(n):
                step()
            for st in [cin, cout] + comp:
                cap.wait_stream(st)
        return g

    run(3)
    steps = max(5, args.steps // 2)
    launch = "eager"
    if not args.eager:
        try:
            g = graph_of(steps)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            g.replay()
            e1.record(main)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            launch = "graph"
        except RuntimeError as ex:  # capture refused: time the same calls eagerly
            launch = f"eager (graph capture failed: {str(ex)[:120]})"
            torch.cuda.synchronize()
    if not launch.startswith("graph"):
        ms = run(steps) / steps
    nr = n_primary + sum(int(ch["count_host"].item()) for ch in chunks)
    h2d = int(rays_host.numel() * 4)
    d2h = int(sum((ch["hits_host"].numel() + ch["hits2_host"].numel()) * 4 + 8 for ch in chunks))
    return {"value": round(world * nr / (ms * 1e-3) / 1e6, 2), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3),
            "steps": steps, "chunks": K, "streams": len(comp),
            "launch": ("all steps replayed from one CUDA graph captured from the API calls"
                       if launch == "graph" else launch),
            "pipeline": "copy-in / trace / copy-out streams ordered by events per slice, "
                        "timed over all steps (no L2 flush: each step moves its rays and hits "
                        "across the host link and walks the whole mesh)"}


# --------------------------------------------------------------------------- #
# CPU oracle (baseline leg and reference arm)


def oracle_step(om, s, W, cam_tet, sel, nthreads, brute=False):
    """One step of the workload on the host oracle for the pixels `sel`; returns rays traced.
    brute: nearest triangle over all of them instead of the walk: the brute-force
    comparison on the tiny scene, and the route for the large scene, whose tet
    adjacency is too large to build on the host."""
    import scenegen as sg
    from oracle.secondary import arrival_side, hit_side, secondary_rays
    o, d = sg.camera_rays(s.camera)
    o, d = o[sel], d[sel]
    if brute:
        w = om.bruteforce(o, d, np.inf, nthreads=nthreads)
        side = arrival_side(s.points, s.tris, w["tri"], d)
    else:
        w = om.trace(o, d, np.inf, cam_tet, nthreads=nthreads)
        ctet = om.ctet_cache if hasattr(om, "ctet_cache") else om.arrays()[2]
        side = hit_side(ctet, w["tri"], w["tet"])
    o2, d2, tm2, entry, _ = secondary_rays(s.points, s.tris, w["tri"], w["b1"], w["b2"], side,
                                           0x5EED, W["per_hit"], W["tmax"], ray_ids=sel)
    if brute:
        om.bruteforce(o2, d2, tm2, exclude=entry >> 1, nthreads=nthreads)
    else:
        om.trace(o2, d2, tm2, -1, entry, nthreads=nthreads)
    return len(o) + len(o2)


def oracle_leg(workload, s, W, frames, tmx, budget_s=20.0):
    """The oracle on the host, after the timed GPU work: its rate on a
    bounded sample (cpu_baseline), then every GPU arm's frame against it
    (vs_oracle).  The rays each arm traced are given to the oracle as they
    are: the primary rays of the camera, and the secondary rays the device
    generated from that arm's own hits, each started from its restart face.
    Where the tet adjacency is too large for the host (the large scene), the
    oracle's brute force over all triangles checks an evenly spaced sample."""
    import oracle
    import scenegen as sg
    from oracle.parity import meets_bar, stats
    nthreads = oracle.default_threads()
    big = s.n_tets > 20_000_000
    om = oracle.OracleTriangles(s.points, s.tris) if big else oracle.OracleMesh(s.points, s.tets, s.tris)
    cpu = cpu_baseline(workload, s, W, budget_s=budget_s, om=om)
    t0 = time.time()
    o, d = sg.camera_rays(s.camera)
    n = len(o)
    if big:
        sel = np.arange(0, n, max(1, n // 2000))
        w1 = om.bruteforce(o[sel], d[sel], np.inf, nthreads=nthreads)
    else:
        sel = np.arange(n)
        cam_tet, _ = om.locate(np.array([s.camera.eye], np.float32), nthreads=nthreads)
        w1 = om.trace(o, d, np.inf, cam_tet[0], nthreads=nthreads)
    out = {}
    for arm, fr in frames.items():
        g1 = tmx.unpack_hits(fr["hits"][sel])
        r2 = fr["rays2"]
        sel2 = np.arange(0, len(r2), max(1, len(r2) // 4000)) if big else np.arange(len(r2))
        r2 = r2[sel2]
        g2 = tmx.unpack_hits(fr["hits2"][sel2])
        entry = -1 - r2.view(np.int32)[:, 3]
        if big:
            w2 = om.bruteforce(r2[:, 0:3], r2[:, 4:7], r2[:, 7], exclude=entry >> 1,
                               nthreads=nthreads)
        else:
            w2 = om.trace(r2[:, 0:3], r2[:, 4:7], r2[:, 7], -1, entry, nthreads=nthreads)
        sp, ss = stats(s.points, s.tris, g1, w1), stats(s.points, s.tris, g2, w2)
        out[arm] = {"primary": sp, "secondary": ss, "meets_bar": meets_bar(sp) and meets_bar(ss),
                    "t_within_1e-5": sp["max_rel_t"] <= 1e-5 and ss["max_rel_t"] <= 1e-5}
    out["sample"] = ("every ray of the frame (primary rays and each arm's device-generated "
                     f"{W['kind']} rays), FP64 face-plane walk"
                     if not big else
                     f"every {max(1, n // 2000)}th primary ray and an even sample of about 4000 "
                     f"{W['kind']} rays per arm, FP64 brute force over all {s.n_tris} triangles")
    out["bar"] = ("ids identical for >= 99.999 % of rays, every mismatch within 1e-6 of a "
                  "triangle edge; t within 1e-5 relative")
    out["oracle_s"] = round(time.time() - t0, 1)
    return cpu, out


def cpu_baseline(workload, s, W, budget_s=20.0, om=None):
    import oracle
    nthreads = oracle.default_threads()
    # a mesh whose tet adjacency is too large to build on the host (the large
    # scene) takes the oracle's brute force over all triangles instead
    big = s.n_tets > 20_000_000
    if big:
        if om is None:
            om = oracle.OracleTriangles(s.points, s.tris)
        cam_tet = [-1]
    else:
        if om is None:
            om = oracle.OracleMesh(s.points, s.tets, s.tris)
        om.ctet_cache = om.arrays()[2]
        cam_tet, _ = om.locate(np.array([s.camera.eye], np.float32), nthreads=nthreads)
    n = s.camera.width * s.camera.height
    stride = 1
    # size the sample: first a small probe, then as many pixels as fit the budget
    probe = np.arange(0, n, max(1, n // (16 if big else 20000)))
    t0 = time.time()
    oracle_step(om, s, W, cam_tet[0], probe, nthreads, brute=big)
    rate = len(probe) / max(time.time() - t0, 1e-6)
    want = int(rate * budget_s)
    if want < n:
        stride = max(1, int(math.ceil(n / max(want, 1))))
    sel = np.arange(0, n, stride)
    t0 = time.time()
    traced = oracle_step(om, s, W, cam_tet[0], sel, nthreads, brute=big)
    dt = time.time() - t0
    if dt < budget_s / 2 and stride > 1:
        # the small probe underestimates the rate: size the sample again from this run
        stride = max(1, int(math.ceil(n / max(1, int(len(sel) / dt * budget_s)))))
        sel = np.arange(0, n, stride)
        t0 = time.time()
        traced = oracle_step(om, s, W, cam_tet[0], sel, nthreads, brute=big)
        dt = time.time() - t0
    passes = 1
    while stride == 1 and dt < budget_s / 2 and passes < 16:
        # the whole frame takes less than the budget: trace it again
        t0 = time.time()
        traced += oracle_step(om, s, W, cam_tet[0], sel, nthreads, brute=big)
        dt += time.time() - t0
        passes += 1
    # the same walk on one core, on a sample 4 x cores times sparser
    stride1 = max(1, stride * nthreads * 4)
    one = np.arange(0, n, stride1)
    t1 = time.time()
    traced1 = oracle_step(om, s, W, cam_tet[0], one, 1, brute=big)
    dt1 = time.time() - t1
    brute = None
    if workload == "tiny":
        # brute force over all triangles, the oracle's other route to the same hits
        allpix = np.arange(n)
        t2 = time.time()
        tb = oracle_step(om, s, W, cam_tet[0], allpix, nthreads, brute=True)
        db = time.time() - t2
        brute = {"value": round(tb / db / 1e6, 4), "unit": UNIT, "cores": nthreads,
                 "sample": f"the whole {s.camera.width}x{s.camera.height} image + its {W['kind']} "
                           f"rays, Moller-Trumbore against all {s.n_tris} triangles; {tb} rays "
                           f"in {db:.2f} s"}
    return {"value": sig4(traced / dt / 1e6), "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{'every' if stride == 1 else f'every {stride}th'} pixel of the {s.camera.width}x{s.camera.height} image "
                      f"({len(sel)} primary rays) + their {W['kind']} rays"
                      + (f", {passes} passes" if passes > 1 else "")
                      + f"; {traced} rays in {dt:.1f} s ("
                      + ("FP64 brute force over all triangles" if big else "FP64 face-plane walk")
                      + ", numpy secondary-ray generation)",
            "single_core": {"value": sig4(traced1 / dt1 / 1e6), "unit": UNIT, "cores": 1,
                            "sample": f"every {stride1}th pixel "
                                      f"({len(one)} primary rays) + their {W['kind']} rays; "
                                      f"{traced1} rays in {dt1:.1f} s"},
            **({"bruteforce": brute} if brute else {})}


def sig4(x):
    """x to four significant digits (the oracle's rates span 1e-4 to 10 Mrays/s)."""
    return float(f"{x:.4g}")


def batched_host_rays(dsc):
    """Host rays of one batched mesh, as its device rays are made: a camera
    grid of about half the rays, then uniform directions from interior points."""
    import scenegen as sg
    n_prim = dsc["primary"]
    side = max(1, int(math.ceil(math.sqrt(n_prim))))
    cam = sg.Camera(sg.BATCHED["camera_eye"], sg.BATCHED["fov_deg"], side,
                    max(1, int(math.ceil(n_prim / side))))
    o1, d1 = sg.camera_rays(cam)
    n_uni = dsc["rays"] - n_prim
    o = np.concatenate([o1, sg.interior_points(n_uni, dsc["seed"])]).astype(np.float32)
    d = np.concatenate([d1, sg.uniform_directions(n_uni, dsc["seed"])]).astype(np.float32)
    return o, d


def run_reference_batched(args):
    """The oracle on the batched workload: every 1024th ray of every mesh per
    step, by brute force over the mesh's triangles (the oracle's route that
    needs no start tet; locating millions of origins on the host would
    dominate)."""
    import oracle
    import scenegen as sg
    nthreads = oracle.default_threads()
    stride = 1024
    work = []
    for dsc in sg.batched_meshes():
        s = sg.make_grid_scene("batched", dsc["n"], sg.BATCHED["jitter"], dsc["seed"],
                               n_spheres=dsc["n_spheres"])
        o, d = batched_host_rays(dsc)
        work.append((oracle.OracleTriangles(s.points, s.tris), o[::stride], d[::stride]))

    def step():
        for ts, o, d in work:
            ts.bruteforce(o, d, np.inf, nthreads=nthreads)
        return sum(len(o) for _, o, _ in work)

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    traced = sum(step() for _ in range(args.steps))
    dt = time.time() - t0
    value = traced / dt / 1e6
    sample = (f"every {stride}th ray of each of the 32 meshes ({traced // args.steps} rays a step), "
              "brute force over the mesh's triangles")
    # "strong", as the GPU arm of this workload reports: its 32 meshes are one
    # fixed job that more ranks split between them, while the single-frame
    # workloads give every replica a whole frame of its own ("weak")
    print(json.dumps({"impl": "reference", "metric": METRIC_BATCHED,
                      "value": sig4(value), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
                      "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"batched: {WORKLOADS['batched']['desc']}",
                                 "mode": "FP64 oracle, brute force"},
                      "cpu_baseline": {"value": sig4(value), "unit": UNIT, "cores": nthreads,
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": sig4(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "batched":
        run_reference_batched(args)
        return
    import oracle
    W = WORKLOADS[args.workload]
    s = build_scene(args.workload)
    nthreads = oracle.default_threads()
    n = s.camera.width * s.camera.height
    # a mesh whose tet adjacency is too large to build on the host (the large
    # scene) takes the oracle's brute force over all triangles instead
    brute = s.n_tets > 20_000_000
    if brute:
        om = oracle.OracleTriangles(s.points, s.tris)
        cam_tet = [-1]
        stride = 16384                            # a bounded sample: every 16384th pixel per step
    else:
        om = oracle.OracleMesh(s.points, s.tets, s.tris)
        om.ctet_cache = om.arrays()[2]
        cam_tet, _ = om.locate(np.array([s.camera.eye], np.float32), nthreads=nthreads)
        stride = 16                               # a bounded sample: every 16th pixel per step
    sel = np.arange(0, n, stride)
    for _ in range(args.warmup):
        oracle_step(om, s, W, cam_tet[0], sel, nthreads, brute=brute)
    t0 = time.time()
    traced = 0
    for _ in range(args.steps):
        traced += oracle_step(om, s, W, cam_tet[0], sel, nthreads, brute=brute)
    dt = time.time() - t0
    value = traced / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": sig4(value), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {W['desc']}",
                       "mode": "FP64 oracle, brute force" if brute else "FP64 oracle walk"},
            "cpu_baseline": {"value": sig4(value), "unit": UNIT, "cores": nthreads,
                             "kind": "oracle",
                             "sample": f"every {stride}th pixel ({len(sel)} primary rays) + their "
                                       f"{W['kind']} rays per step"
                                       + (", brute force over all triangles" if brute else "")},
            "e2e": {"value": sig4(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, world, rank, local):
    """32 uneven meshes: one persistent graph-replayed launch vs 32 separate launches.

    With N ranks the meshes are split by longest-processing-time on their
    estimated cost (rays x grid cells per axis, the walk length scale); each
    rank traces its share and the step time is the slowest rank's."""
    import torch
    from paper_2103_02309_gb300 import build as libbuild
    if rank == 0 or not os.path.exists(libbuild.LIB):
        libbuild.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import scenegen as sg
    from paper_2103_02309_gb300 import tetmesh as tmx
    from paper_2103_02309_gb300.shard import lpt_assign, max_over_ranks
    dev = torch.device("cuda", local)
    all_descs = sg.batched_meshes()
    owner = lpt_assign([d["rays"] * d["n"] for d in all_descs], world)
    descs = [d for d, r in zip(all_descs, owner) if r == rank]
    total_all = sum(d["rays"] for d in all_descs)
    meshes, rays, hits = [], [], []
    t0 = time.time()
    for dsc in descs:
        s = sg.make_grid_scene("batched", dsc["n"], sg.BATCHED["jitter"], dsc["seed"],
                               n_spheres=dsc["n_spheres"])
        mesh = tmx.Mesh(s.points, s.tets, s.tris, faces=True, faces16=True)
        n_prim = dsc["primary"]
        side = max(1, int(math.ceil(math.sqrt(n_prim))))
        cam = tmx.make_camera(sg.BATCHED["camera_eye"], sg.BATCHED["fov_deg"], side,
                              max(1, int(math.ceil(n_prim / side))))
        eye = torch.tensor([sg.BATCHED["camera_eye"]], dtype=torch.float32, device=dev)
        r1 = tmx.gen_primary(cam, mesh.locate(eye))
        n_uni = dsc["rays"] - n_prim
        q = torch.from_numpy(sg.interior_points(n_uni, dsc["seed"])).to(dev)
        tet = mesh.locate(q)
        d = sg.uniform_directions(n_uni, dsc["seed"])
        r2 = torch.empty((n_uni, 8), dtype=torch.float32, device=dev)
        r2[:, 0:3] = q
        r2[:, 4:7] = torch.from_numpy(d).to(dev)
        r2[:, 7] = float("inf")
        r2.view(torch.int32)[:, 3] = tet
        r = torch.cat([r1, r2]).contiguous()
        meshes.append(mesh)
        rays.append(r)
        hits.append(torch.empty((r.shape[0], 8), dtype=torch.int32, device=dev))
    build_s = time.time() - t0
    total = sum(int(r.shape[0]) for r in rays)
    b = tmx.Batch(meshes)
    b.set(rays, hits)
    tuned = b.autotune(reps=2)
    stream = torch.cuda.current_stream()

    def timeit(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        l0 = tmx.launch_count()
        tot = 0.0
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps, tmx.launch_count() - l0

    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        ms_graph, launches = timeit(b.run, args.steps)
    ms_sep, _ = timeit(b.run_separate, args.steps)
    if world > 1:
        torch.distributed.barrier()
    ms_graph = max_over_ranks(ms_graph, dev)
    ms_sep = max_over_ranks(ms_sep, dev)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    total = total_all
    value = total / (ms_graph * 1e-3) / 1e6
    line = {"metric": METRIC_BATCHED, "value": round(value, 2),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 3,
            "ms_per_step": round(ms_graph, 3), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched: {WORKLOADS['batched']['desc']}", "rays": total,
                       "meshes": len(all_descs), "meshes_rank0": len(meshes),
                       "parallelism": f"replicas x{world}, meshes split by LPT" if world > 1 else "1 GPU", "tets": int(sum(m.n_tets for m in meshes)),
                       "build_s": round(build_s, 1),
                       "autotuned": {"format": {v: k for k, v in tmx.FORMATS.items()}[tuned.opts.format],
                                     "block": tuned.opts.block, "refill": tuned.opts.refill,
                                     "batch_steps": tuned.opts.batch_steps,
                                     "sort_chunk": tuned.sort_chunk, "ms": round(tuned.ms, 3)}},
            "separate_launches": {"value": round(total / (ms_sep * 1e-3) / 1e6, 2),
                                  "ms_per_step": round(ms_sep, 3)},
            "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
