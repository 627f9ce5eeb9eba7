"""ctypes bindings of libtetmesh.so (include/tetmesh.h).  Argument marshalling
only: every step of the traversal runs in the library's CUDA kernels.

Importing this module loads the library and raises ImportError when it is
missing or cannot be loaded; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB


class NativeLibraryMissing(ImportError):
    pass


def _load():
    path = os.environ.get("TETMESH_LIB", LIB_PATH)
    if not os.path.exists(path):
        raise NativeLibraryMissing(
            f"{path} is missing: build it with `python -m paper_2103_02309_gb300.build` "
            "(or __graft_entry__.build()); the library has no non-CUDA fallback")
    try:
        return ctypes.CDLL(path)
    except OSError as e:
        raise NativeLibraryMissing(f"cannot load {path}: {e}") from e


lib = _load()

P = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
u64 = ctypes.c_uint64
f32 = ctypes.c_float
f64 = ctypes.c_double


class BuildOpts(ctypes.Structure):
    _fields_ = [("order", i32), ("fix_orientation", i32), ("tet20", i32), ("faces", i32),
                ("faces16", i32)]


class TraceOpts(ctypes.Structure):
    _fields_ = [("mode", i32), ("guard_tau", f32), ("max_steps", ctypes.c_uint32), ("block", i32),
                ("refill", i32), ("batch_steps", i32), ("ctas_per_sm", i32),
                ("tmax_early_exit", i32), ("phase_events", P * 4), ("format", i32)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_points", i64), ("n_tets", i64), ("n_tris", i64), ("extent", f64),
                ("bbox_lo", f32 * 3), ("bbox_hi", f32 * 3), ("source_tet", i32),
                ("on_device", i32), ("tet16_dev", P), ("points_dev", P), ("cold_dev", P),
                ("cface_dev", P), ("tet20_dev", P), ("tet20_n3_dev", P), ("tet20_aos_dev", P), ("face_dev", P), ("face16_dev", P),
                ("device_bytes", i64), ("n_regions", i64)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", f32 * 3), ("width", i32), ("height", i32), ("kx", f32), ("ky", f32),
                ("tx", f32), ("ty", f32)]


class Tuned(ctypes.Structure):
    _fields_ = [("opts", TraceOpts), ("sort_chunk", i32), ("ms", f32)]


_SIGS = {
    "tm_build": ([P, i64, P, i64, P, i64, ctypes.POINTER(BuildOpts), ctypes.c_int,
                  ctypes.POINTER(P)], ctypes.c_int),
    "tm_destroy": ([P], None),
    "tm_mesh_info_get": ([P, ctypes.POINTER(MeshInfo)], ctypes.c_int),
    "tm_mesh_export": ([P, P, P, P, P, P, P], ctypes.c_int),
    "tm_mesh_export_tet20": ([P, P, P, P], ctypes.c_int),
    "tm_mesh_export_faces": ([P, P], ctypes.c_int),
    "tm_mesh_export_faces16": ([P, P], ctypes.c_int),
    "tm_mesh_export_restart": ([P, P], ctypes.c_int),
    "tm_map_ids": ([P, ctypes.c_int, ctypes.c_int, P, P, i64], ctypes.c_int),
    "tm_hilbert_keys": ([P, i64, ctypes.c_int, P], ctypes.c_int),
    "tm_locate": ([P, P, i64, P, i32, P, P], ctypes.c_int),
    "tm_trace": ([P, P, i64, P, P, ctypes.POINTER(TraceOpts), P], ctypes.c_int),
    "tm_trace_shadow": ([P, P, i64, P, P, P, ctypes.POINTER(TraceOpts), P], ctypes.c_int),
    "tm_gen_primary": ([ctypes.POINTER(Camera), P, f32, P, P], ctypes.c_int),
    "tm_gen_secondary": ([P, P, i64, P, ctypes.c_int, f32, u64, P, P, P, P], ctypes.c_int),
    "tm_gen_shadow": ([P, P, i64, P, f32, f32, f32, P, P, P, P], ctypes.c_int),
    "tm_gen_specular": ([P, P, P, i64, P, ctypes.c_int, f32, f32, P, P, P, P], ctypes.c_int),
    "tm_gen_secondary_noalloc": ([P, P, i64, P, ctypes.c_int, f32, u64, P, P, P, P], ctypes.c_int),
    "tm_batch_create": ([P, ctypes.c_int, ctypes.POINTER(P)], ctypes.c_int),
    "tm_batch_set": ([P, P, P, P, ctypes.POINTER(TraceOpts), i32], ctypes.c_int),
    "tm_batch_run": ([P, P], ctypes.c_int),
    "tm_batch_run_separate": ([P, P], ctypes.c_int),
    "tm_batch_autotune": ([P, ctypes.c_int, ctypes.POINTER(Tuned), P], ctypes.c_int),
    "tm_batch_destroy": ([P], None),
    "tm_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "tm_last_error": ([], ctypes.c_char_p),
    "tm_launch_count": ([], ctypes.c_uint64),
}

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class TetmeshError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.tm_status_str(status).decode()
        if status == 8:
            msg += ": " + lib.tm_last_error().decode()
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != 0:
        raise TetmeshError(status, where)
