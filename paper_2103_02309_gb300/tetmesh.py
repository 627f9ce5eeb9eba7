"""Python front end of the tet-mesh ray traversal library.

Rays and hits live in CUDA tensors laid out as the C structs of
include/tetmesh.h (32 bytes each): rays as float32 [n, 8]
(ox, oy, oz, start-as-int32-bits, dx, dy, dz, tmax), hits as int32 [n, 8]
(tri, t-bits, b1-bits, b2-bits, tet, cface, steps, flags).  PyTorch only
provides device memory and the current stream; the work runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native as N

MODES = {"fp32g": 0, "fp32": 1, "fp64": 2}
FORMATS = {"auto": 0, "tet16": 1, "tet20": 2, "tet32": 3, "tet20_aos": 4, "face": 5, "face16": 6}
ORDERS = {"hilbert": 0, "input": 1, "hilbert_regions": 2}

HIT_SIDE_NEG = 0x01
HIT_STEP_LIMIT = 0x02
HIT_GUARD = 0x04
HIT_BAD_START = 0x08
HIT_TIE = 0x10
HIT_FINAL_FP64 = 0x20
HIT_RESTART_3D = 0x40
HIT_BAD_ID = 0x80
HIT_START_MOVED = 0x100
HIT_SLOW_PASS = 0x200
HIT_REACHED = 0x400
SPECULAR = {"reflect": 0, "refract": 1}

IDS_TET, IDS_POINT = 0, 1
TO_INPUT, TO_INTERNAL = 0, 1


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def trace_opts(mode="fp32g", guard_tau=0.0, max_steps=0, block=0, refill=0, batch_steps=0,
               ctas_per_sm=0, tmax_early_exit=False, phase_events=None, format="auto") -> N.TraceOpts:
    """Trace options; phase_events: four torch.cuda.Event (enable_timing) recorded
    before the start phase, after it, after the walk and after the finish phase."""
    o = N.TraceOpts()
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.guard_tau = float(guard_tau)
    o.max_steps = int(max_steps)
    o.block = int(block)
    o.refill = int(refill)
    o.batch_steps = int(batch_steps)
    o.ctas_per_sm = int(ctas_per_sm)
    o.tmax_early_exit = 1 if tmax_early_exit else 0
    o.format = FORMATS[format] if isinstance(format, str) else int(format)
    if phase_events is not None:
        for i, ev in enumerate(phase_events):
            o.phase_events[i] = ev.cuda_event if ev is not None else None
    return o


def pack_rays(o, d, tmax, start) -> np.ndarray:
    """Host float32 [n, 8] ray records (see the module doc)."""
    o = np.asarray(o, np.float32).reshape(-1, 3)
    n = len(o)
    r = np.empty((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = np.asarray(d, np.float32).reshape(-1, 3)
    r[:, 7] = np.broadcast_to(np.asarray(tmax, np.float32), (n,))
    r.view(np.int32)[:, 3] = np.broadcast_to(np.asarray(start, np.int32), (n,))
    return r


def restart_start(tri, side):
    """tm_ray.start value of a ray restarted from triangle `tri` into its `side`."""
    return -1 - (2 * np.asarray(tri, np.int64) + np.asarray(side, np.int64))


def unpack_hits(h) -> dict:
    """Hits (CUDA or host int32 [n, 8]) as a dict of host numpy arrays."""
    a = h.cpu().numpy() if isinstance(h, torch.Tensor) else np.asarray(h)
    a = np.ascontiguousarray(a, dtype=np.int32).reshape(-1, 8)
    f = a.view(np.float32)
    return dict(tri=a[:, 0].copy(), t=f[:, 1].copy(), b1=f[:, 2].copy(), b2=f[:, 3].copy(),
                tet=a[:, 4].copy(), cface=a[:, 5].copy(), steps=a[:, 6].view(np.uint32).copy(),
                flags=a[:, 7].view(np.uint32).copy())


def make_camera(eye, fov_deg, width, height) -> N.Camera:
    """Pinhole camera of the synthetic workloads (looking along +z); the float32
    constants are computed in float64 and rounded once."""
    c = N.Camera()
    for i in range(3):
        c.eye[i] = float(eye[i])
    c.width, c.height = int(width), int(height)
    short = min(width, height)
    tanh = math.tan(math.radians(fov_deg) * 0.5)
    c.kx, c.ky = 2.0 / width, 2.0 / height
    c.tx, c.ty = tanh * (width / short), tanh * (height / short)
    return c


class Mesh:
    """A compact constrained tet mesh on the current CUDA device."""

    def __init__(self, points, tets, tris, order="hilbert", upload=True, fix_orientation=False,
                 tet20=False, faces=False, faces16=False):
        pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
        tt = np.ascontiguousarray(tets, np.int32).reshape(-1, 4)
        tr = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        o = N.BuildOpts(ORDERS[order], 1 if fix_orientation else 0, 1 if tet20 else 0,
                        1 if faces else 0, 1 if faces16 else 0)
        h = ctypes.c_void_p()
        N.check(N.lib.tm_build(_hptr(pts), len(pts), _hptr(tt), len(tt),
                               _hptr(tr) if len(tr) else None, len(tr), ctypes.byref(o),
                               1 if upload else 0, ctypes.byref(h)), "tm_build")
        self._h = h
        self.n_points, self.n_tets, self.n_tris = len(pts), len(tt), len(tr)

    def close(self):
        if getattr(self, "_h", None):
            N.lib.tm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def info(self) -> N.MeshInfo:
        i = N.MeshInfo()
        N.check(N.lib.tm_mesh_info_get(self._h, ctypes.byref(i)), "tm_mesh_info_get")
        return i

    def export(self) -> dict:
        nt, np_, nc = self.n_tets, self.n_points, self.n_tris
        out = dict(tet16=np.empty((nt, 4), np.int32), cold=np.empty((nt, 8), np.int32),
                   points=np.empty((np_, 4), np.float32), cface=np.empty((max(nc, 1), 8), np.int32),
                   point_perm=np.empty(np_, np.int32), tet_perm=np.empty(nt, np.int32))
        N.check(N.lib.tm_mesh_export(self._h, *[_hptr(out[k]) for k in
                                                ("tet16", "cold", "points", "cface",
                                                 "point_perm", "tet_perm")]), "tm_mesh_export")
        out["cface"] = out["cface"][:nc]
        return out

    def export_tet20(self) -> dict:
        vxn = np.empty((self.n_tets, 4), np.int32)
        n3 = np.empty(self.n_tets, np.int32)
        aos = np.empty((self.n_tets, 5), np.int32)
        N.check(N.lib.tm_mesh_export_tet20(self._h, _hptr(vxn), _hptr(n3), _hptr(aos)),
                "tm_mesh_export_tet20")
        return dict(vxn=vxn, n3=n3, aos=aos)

    def export_faces(self) -> np.ndarray:
        """Face entries int32 [n_tets, 4, 8] (see TM_FORMAT_FACE)."""
        f = np.empty((self.n_tets, 4, 8), np.int32)
        N.check(N.lib.tm_mesh_export_faces(self._h, _hptr(f)), "tm_mesh_export_faces")
        return f

    def export_faces16(self) -> np.ndarray:
        """16-byte face entries int32 [n_tets, 4, 4] (see TM_FORMAT_FACE16)."""
        f = np.empty((self.n_tets, 4, 4), np.int32)
        N.check(N.lib.tm_mesh_export_faces16(self._h, _hptr(f)), "tm_mesh_export_faces16")
        return f

    def export_restart(self) -> np.ndarray:
        """Restart records int32 [n_tris, 2, 24] (see tm_mesh_export_restart)."""
        r = np.empty((max(self.info.n_tris, 0), 2, 24), np.int32)
        N.check(N.lib.tm_mesh_export_restart(self._h, _hptr(r)), "tm_mesh_export_restart")
        return r

    def map_ids(self, kind, direction, ids) -> np.ndarray:
        a = np.ascontiguousarray(ids, np.int32).reshape(-1)
        out = np.empty_like(a)
        N.check(N.lib.tm_map_ids(self._h, kind, direction, _hptr(a), _hptr(out), len(a)),
                "tm_map_ids")
        return out

    def locate(self, q: torch.Tensor, hint: torch.Tensor | None = None, source: int = -1,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        q = q.contiguous()
        n = q.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=q.device)
        N.check(N.lib.tm_locate(self._h, _dptr(q), n, _dptr(hint), int(source), _dptr(out),
                                _stream(stream)), "tm_locate")
        return out

    def trace(self, rays: torch.Tensor, hits: torch.Tensor | None = None,
              n_dev: torch.Tensor | None = None, opts: N.TraceOpts | None = None, stream=None,
              **kw) -> torch.Tensor:
        n = rays.shape[0]
        if hits is None:
            hits = torch.empty((n, 8), dtype=torch.int32, device=rays.device)
        o = opts if opts is not None else trace_opts(**kw)
        N.check(N.lib.tm_trace(self._h, _dptr(rays), n, _dptr(n_dev), _dptr(hits),
                               ctypes.byref(o), _stream(stream)), "tm_trace")
        return hits

    def trace_shadow(self, rays: torch.Tensor, light_tet: torch.Tensor,
                     hits: torch.Tensor | None = None, n_dev: torch.Tensor | None = None,
                     opts: N.TraceOpts | None = None, stream=None, **kw) -> torch.Tensor:
        """Walks that also end (flag HIT_REACHED) on entering the light's tet
        (light_tet: device int32 tensor, e.g. from locate)."""
        n = rays.shape[0]
        if hits is None:
            hits = torch.empty((n, 8), dtype=torch.int32, device=rays.device)
        o = opts if opts is not None else trace_opts(**kw)
        N.check(N.lib.tm_trace_shadow(self._h, _dptr(rays), n, _dptr(n_dev), _dptr(light_tet),
                                      _dptr(hits), ctypes.byref(o), _stream(stream)),
                "tm_trace_shadow")
        return hits

    def _outputs(self, n, device, rays_out, count, src):
        if rays_out is None:
            rays_out = torch.empty((n, 8), dtype=torch.float32, device=device)
        if count is None:
            count = torch.empty(1, dtype=torch.int64, device=device)
        if src is True:
            src = torch.empty(n, dtype=torch.int32, device=device)
        elif src is False:
            src = None
        return rays_out, count, src

    def gen_shadow(self, hits: torch.Tensor, light, n_dev: torch.Tensor | None = None,
                   rays_out: torch.Tensor | None = None, count: torch.Tensor | None = None,
                   src: bool | torch.Tensor = False, stream=None):
        n = hits.shape[0]
        rays_out, count, src = self._outputs(n, hits.device, rays_out, count, src)
        lx, ly, lz = (float(v) for v in light)
        N.check(N.lib.tm_gen_shadow(self._h, _dptr(hits), n, _dptr(n_dev), lx, ly, lz,
                                    _dptr(rays_out), _dptr(count), _dptr(src), _stream(stream)),
                "tm_gen_shadow")
        return rays_out, count, src

    def gen_specular(self, rays_in: torch.Tensor, hits: torch.Tensor, kind: str, ior: float,
                     tmax: float = float("inf"), n_dev: torch.Tensor | None = None,
                     rays_out: torch.Tensor | None = None, count: torch.Tensor | None = None,
                     src: bool | torch.Tensor = False, stream=None):
        n = hits.shape[0]
        rays_out, count, src = self._outputs(n, hits.device, rays_out, count, src)
        k = SPECULAR[kind] if isinstance(kind, str) else int(kind)
        N.check(N.lib.tm_gen_specular(self._h, _dptr(rays_in), _dptr(hits), n, _dptr(n_dev), k,
                                      float(ior), float(tmax), _dptr(rays_out), _dptr(count),
                                      _dptr(src), _stream(stream)), "tm_gen_specular")
        return rays_out, count, src

    def gen_secondary(self, hits: torch.Tensor, per_hit: int, tmax: float, seed: int,
                      n_dev: torch.Tensor | None = None, rays_out: torch.Tensor | None = None,
                      count: torch.Tensor | None = None, src: bool | torch.Tensor = False,
                      stream=None):
        n = hits.shape[0]
        if rays_out is None:
            rays_out = torch.empty((n * per_hit, 8), dtype=torch.float32, device=hits.device)
        if count is None:
            count = torch.empty(1, dtype=torch.int64, device=hits.device)
        if src is True:
            src = torch.empty(n * per_hit, dtype=torch.int32, device=hits.device)
        elif src is False:
            src = None
        N.check(N.lib.tm_gen_secondary(self._h, _dptr(hits), n, _dptr(n_dev), int(per_hit),
                                       float(tmax), int(seed) & ((1 << 64) - 1), _dptr(rays_out),
                                       _dptr(count), _dptr(src), _stream(stream)),
                "tm_gen_secondary")
        return rays_out, count, src


def gen_primary(cam: N.Camera, start_dev: torch.Tensor, tmax: float = float("inf"),
                rays: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = cam.width * cam.height
    if rays is None:
        rays = torch.empty((n, 8), dtype=torch.float32, device=start_dev.device)
    N.check(N.lib.tm_gen_primary(ctypes.byref(cam), _dptr(start_dev), float(tmax), _dptr(rays),
                                 _stream(stream)), "tm_gen_primary")
    return rays


def hilbert_keys(ijk, bits: int) -> np.ndarray:
    a = np.ascontiguousarray(ijk, np.uint32).reshape(-1, 3)
    out = np.empty(len(a), np.uint64)
    N.check(N.lib.tm_hilbert_keys(_hptr(a), len(a), int(bits), _hptr(out)), "tm_hilbert_keys")
    return out


def launch_count() -> int:
    return int(N.lib.tm_launch_count())


class Batch:
    """Many meshes traced in one persistent launch replayed from a CUDA graph."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        h = ctypes.c_void_p()
        N.check(N.lib.tm_batch_create(arr, len(self.meshes), ctypes.byref(h)), "tm_batch_create")
        self._h = h
        self._keep = None

    def set(self, rays, hits, opts: N.TraceOpts | None = None, sort_chunk: int = 0, **kw):
        k = len(self.meshes)
        ra = (ctypes.c_void_p * k)(*[r.data_ptr() for r in rays])
        ha = (ctypes.c_void_p * k)(*[h.data_ptr() for h in hits])
        na = (ctypes.c_int64 * k)(*[r.shape[0] for r in rays])
        o = opts if opts is not None else trace_opts(**kw)
        N.check(N.lib.tm_batch_set(self._h, ra, na, ha, ctypes.byref(o), int(sort_chunk)),
                "tm_batch_set")
        self._keep = (rays, hits)

    def run(self, stream=None):
        N.check(N.lib.tm_batch_run(self._h, _stream(stream)), "tm_batch_run")

    def run_separate(self, stream=None):
        N.check(N.lib.tm_batch_run_separate(self._h, _stream(stream)), "tm_batch_run_separate")

    def autotune(self, reps=3, stream=None) -> N.Tuned:
        t = N.Tuned()
        N.check(N.lib.tm_batch_autotune(self._h, int(reps), ctypes.byref(t), _stream(stream)),
                "tm_batch_autotune")
        return t

    def close(self):
        if getattr(self, "_h", None):
            N.lib.tm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
