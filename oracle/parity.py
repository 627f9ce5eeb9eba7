"""Comparison of CUDA hits against the FP64 oracle: the parity bar of the
GPU tests, the smoke check and the benchmark's oracle leg.  Test
infrastructure, like the rest of this package.

Tolerances (the parity bar of this project, scene extent E = 1):
* triangle id identical for >= 99.999 % of rays; a mismatch is excused only
  when the hit that one side reports lies within 1e-6 * E of an edge of its
  triangle (the near-edge tie of the two arithmetics);
* t within 1e-5 relative error (FP32 with FP64 guard, and FP64);
* the hit point (1-b1-b2) v0 + b1 v1 + b2 v2 within 2e-6 * E * max(1, t).
"""
from __future__ import annotations

import numpy as np

ID_AGREEMENT = 0.99999
T_RTOL = 1e-5
EDGE_TOL = 1e-6
POINT_TOL = 2e-6


def edge_distance(points, tris, tri, b1, b2):
    """Distance (scene units) of the point with barycentrics (b1, b2) from its triangle's edges."""
    P = np.asarray(points, np.float64)
    tri = np.asarray(tri)
    v0, v1, v2 = P[tris[tri, 0]], P[tris[tri, 1]], P[tris[tri, 2]]
    b1 = np.asarray(b1, np.float64)
    b2 = np.asarray(b2, np.float64)
    b0 = 1.0 - b1 - b2

    def height(a, b, c):  # distance of c from the line through a, b
        ab = b - a
        return np.linalg.norm(np.cross(ab, c - a), axis=1) / np.linalg.norm(ab, axis=1)
    # barycentric of vertex k times the vertex's height over the opposite edge
    return np.minimum.reduce([np.abs(b0) * height(v1, v2, v0), np.abs(b1) * height(v2, v0, v1),
                              np.abs(b2) * height(v0, v1, v2)])


def hit_points(points, tris, tri, b1, b2):
    P = np.asarray(points, np.float64)
    v0, v1, v2 = P[tris[tri, 0]], P[tris[tri, 1]], P[tris[tri, 2]]
    b1 = np.asarray(b1, np.float64)[:, None]
    b2 = np.asarray(b2, np.float64)[:, None]
    return (1.0 - b1 - b2) * v0 + b1 * v1 + b2 * v2


def stats(points, tris, gpu: dict, orc: dict) -> dict:
    """Agreement of GPU hits with the oracle's, without asserting anything:
    id agreement, mismatches and how many are not excused by the near-edge
    rule, t errors (max, p99) and hit-point errors on agreeing hits, and the
    miss/hit confusions."""
    g_tri, o_tri = np.asarray(gpu["tri"]), np.asarray(orc["tri"])
    n = len(g_tri)
    same = g_tri == o_tri
    bad = np.nonzero(~same)[0]
    excused = np.zeros(len(bad), bool)
    if len(bad):
        oh = o_tri[bad] >= 0
        gh = g_tri[bad] >= 0
        near_o = np.zeros(len(bad), bool)
        near_g = np.zeros(len(bad), bool)
        if oh.any():
            near_o[oh] = edge_distance(points, tris, o_tri[bad][oh], orc["b1"][bad][oh],
                                       orc["b2"][bad][oh]) < EDGE_TOL
        if gh.any():
            near_g[gh] = edge_distance(points, tris, g_tri[bad][gh], gpu["b1"][bad][gh],
                                       gpu["b2"][bad][gh]) < EDGE_TOL
        excused = near_o | near_g
    both = same & (g_tri >= 0)
    rel = np.zeros(0)
    perr = np.zeros(0)
    if both.any():
        ot = np.asarray(orc["t"], np.float64)[both]
        rel = np.abs(np.asarray(gpu["t"], np.float64)[both] - ot) / np.maximum(np.abs(ot), 1e-30)
        xg = hit_points(points, tris, g_tri[both], gpu["b1"][both], gpu["b2"][both])
        xo = hit_points(points, tris, o_tri[both], orc["b1"][both], orc["b2"][both])
        perr = np.linalg.norm(xg - xo, axis=1) / np.maximum(1.0, np.abs(ot))
    return dict(n=n, agree=float(same.mean()) if n else 1.0, mismatches=int(len(bad)),
                unexcused=int((~excused).sum()), hits=int((o_tri >= 0).sum()),
                max_rel_t=float(rel.max()) if len(rel) else 0.0,
                p99_rel_t=float(np.percentile(rel, 99)) if len(rel) else 0.0,
                max_point_err=float(perr.max()) if len(perr) else 0.0,
                miss_hit=int(((g_tri < 0) & (o_tri >= 0)).sum()),
                hit_miss=int(((g_tri >= 0) & (o_tri < 0)).sum()))


def meets_bar(st: dict) -> bool:
    """Every mismatch excused and at least 99.999 % of ids identical (one
    excused mismatch allowed for small batches)."""
    return (st["unexcused"] == 0
            and st["mismatches"] <= max(1, int(np.ceil((1 - ID_AGREEMENT) * st["n"]))))


def compare(points, tris, gpu: dict, orc: dict, t_rtol=T_RTOL, check_t=True, rate_bar=True):
    """Returns a stats dict; raises AssertionError when the bar is not met.
    rate_bar=False keeps every other check but not the 99.999 % agreement
    rate, for inputs built to put hits exactly on triangle edges, where
    every mismatch is an excused tie."""
    st = stats(points, tris, gpu, orc)
    # every mismatch excused, and at least 99.999 % identical (at least one
    # excused mismatch allowed for small batches)
    assert st["unexcused"] == 0, st
    if rate_bar:
        assert meets_bar(st), st
    if check_t:
        assert st["max_rel_t"] <= t_rtol, st
        assert st["max_point_err"] <= POINT_TOL, st
    return st
