"""FP64 CPU oracle for constrained tet-mesh ray traversal.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg and its reference arm.  The product path never
imports it.  It shares no code with the CUDA library; see oracle.c for the
definition of the result it computes and how.

Parity pins (tests/test_oracle_pins.py) tie it to the geometry: brute force
over all triangles, closed-form plane and sphere hits, mesh invariants and
exhaustive checks on tiny meshes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_STEP_LIMIT = 1
FLAG_DEGENERATE = 2
FLAG_BAD_START = 4
FLAG_NONMONOTONE = 8
FLAG_TIE = 16


def build(src: str = _SRC, out: str = _LIB_PATH, defines=()) -> str:
    """Compile oracle.c with gcc (plain C, IEEE double, no contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", out, src, "-lpthread", "-lm"]
    cmd += [f"-D{d}" for d in defines]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.orc_mesh_create.argtypes = [i64, P, i64, P, i64, P, ctypes.POINTER(P)]
    lib.orc_mesh_create.restype = ctypes.c_int
    lib.orc_mesh_destroy.argtypes = [P]
    lib.orc_soup_create.argtypes = [i64, P, i64, P, ctypes.POINTER(P)]
    lib.orc_soup_create.restype = ctypes.c_int
    lib.orc_mesh_arrays.argtypes = [P, P, P, P]
    for f in ("orc_count_nonpositive", "orc_count_asymmetric", "orc_count_boundary"):
        getattr(lib, f).argtypes = [P]
        getattr(lib, f).restype = i64
    lib.orc_trace.argtypes = [P, i64, P, P, P, P, P, i64, ctypes.c_int] + [P] * 8
    lib.orc_bruteforce.argtypes = [P, i64, P, P, P, P, ctypes.c_int] + [P] * 4
    lib.orc_locate.argtypes = [P, i64, P, ctypes.c_int, P, P]
    lib.orc_tet_bary.argtypes = [P, ctypes.c_int32, P, P]
    lib.orc_mesh_relink.argtypes = [P, i64, ctypes.c_int, ctypes.c_int32, ctypes.c_int]
    lib.orc_mesh_relink.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(_LIB_PATH)
                     or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
            if stale:
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


class OracleError(RuntimeError):
    pass


_STATUS = {1: "bad argument or id out of range", 2: "a face is shared by more than two tets",
           3: "a constrained triangle is not a tet face", 4: "two triangles on one tet face",
           5: "out of memory"}


class OracleMesh:
    """Points (float32 [np,3]), tets (int32 [nt,4], positively oriented), triangles (int32 [nc,3])."""

    def __init__(self, points, tets, tris, lib=None):
        self.lib = lib or load()
        self.points = np.ascontiguousarray(points, dtype=np.float32)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        h = ctypes.c_void_p()
        st = self.lib.orc_mesh_create(len(self.points), _ptr(self.points), len(self.tets),
                                      _ptr(self.tets), len(self.tris), _ptr(self.tris),
                                      ctypes.byref(h))
        if st != 0:
            raise OracleError(_STATUS.get(st, f"status {st}"))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.orc_mesh_destroy(h)
            self._h = None

    @property
    def n_tets(self):
        return len(self.tets)

    def arrays(self):
        nbr = np.empty((self.n_tets, 4), np.int32)
        fc = np.empty((self.n_tets, 4), np.int32)
        ctet = np.empty((max(len(self.tris), 1), 2), np.int32)
        self.lib.orc_mesh_arrays(self._h, _ptr(nbr), _ptr(fc), _ptr(ctet))
        return nbr, fc, ctet[: len(self.tris)]

    def count_nonpositive(self):
        return int(self.lib.orc_count_nonpositive(self._h))

    def count_asymmetric(self):
        return int(self.lib.orc_count_asymmetric(self._h))

    def count_boundary(self):
        return int(self.lib.orc_count_boundary(self._h))

    def relink(self, t, k, u, ku):
        """Test hook: overwrite the link of tet t across face k with (u, ku)."""
        if self.lib.orc_mesh_relink(self._h, int(t), int(k), int(u), int(ku)) != 0:
            raise OracleError("relink: bad arguments")

    def trace(self, o, d, tmax, start, entry=None, max_steps=None, nthreads=None):
        """Definitional FP64 walk.  entry = 2*c + side restarts through triangle c (else -1)."""
        o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
        n = len(o)
        tmax = np.ascontiguousarray(np.broadcast_to(np.asarray(tmax, np.float32), (n,)))
        start = np.ascontiguousarray(np.broadcast_to(np.asarray(start, np.int32), (n,)))
        entry = np.full(n, -1, np.int32) if entry is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(entry, np.int32), (n,)))
        out = dict(tri=np.empty(n, np.int32), t=np.empty(n), b1=np.empty(n), b2=np.empty(n),
                   tet=np.empty(n, np.int32), cface=np.empty(n, np.int32),
                   steps=np.empty(n, np.int32), flags=np.empty(n, np.int32))
        ms = max_steps if max_steps is not None else 16 * self.n_tets + 64
        self.lib.orc_trace(self._h, n, _ptr(o), _ptr(d), _ptr(tmax), _ptr(start), _ptr(entry),
                           ms, nthreads or default_threads(),
                           _ptr(out["tri"]), _ptr(out["t"]), _ptr(out["b1"]), _ptr(out["b2"]),
                           _ptr(out["tet"]), _ptr(out["cface"]), _ptr(out["steps"]),
                           _ptr(out["flags"]))
        return out

    def bruteforce(self, o, d, tmax, exclude=None, nthreads=None):
        o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
        n = len(o)
        tmax = np.ascontiguousarray(np.broadcast_to(np.asarray(tmax, np.float32), (n,)))
        exclude = np.full(n, -1, np.int32) if exclude is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(exclude, np.int32), (n,)))
        out = dict(tri=np.empty(n, np.int32), t=np.empty(n), b1=np.empty(n), b2=np.empty(n))
        self.lib.orc_bruteforce(self._h, n, _ptr(o), _ptr(d), _ptr(tmax), _ptr(exclude),
                                nthreads or default_threads(), _ptr(out["tri"]), _ptr(out["t"]),
                                _ptr(out["b1"]), _ptr(out["b2"]))
        return out

    def locate(self, q, nthreads=None):
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, 3)
        tet = np.empty(len(q), np.int32)
        mb = np.empty(len(q))
        self.lib.orc_locate(self._h, len(q), _ptr(q), nthreads or default_threads(), _ptr(tet),
                            _ptr(mb))
        return tet, mb

    def tet_bary(self, t, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        w = np.empty(4)
        self.lib.orc_tet_bary(self._h, int(t), _ptr(q), _ptr(w))
        return w


class OracleTriangles(OracleMesh):
    """Points and triangles without tets: only `bruteforce` (the plain
    definition of the hit, nearest triangle over all of them) is available.
    For scenes whose tet adjacency is too large to build on the host."""

    def __init__(self, points, tris, lib=None):
        self.lib = lib or load()
        self.points = np.ascontiguousarray(points, dtype=np.float32)
        self.tets = np.zeros((0, 4), np.int32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        h = ctypes.c_void_p()
        st = self.lib.orc_soup_create(len(self.points), _ptr(self.points), len(self.tris),
                                      _ptr(self.tris), ctypes.byref(h))
        if st != 0:
            raise OracleError(_STATUS.get(st, f"status {st}"))
        self._h = h

    def _tetless(self, *a, **k):
        raise OracleError("a triangle set has no tets")

    trace = locate = arrays = tet_bary = relink = _tetless
    count_nonpositive = count_asymmetric = count_boundary = _tetless
