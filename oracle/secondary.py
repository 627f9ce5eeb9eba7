"""Secondary rays from hits, FP64 (test infrastructure; see oracle/__init__.py).

Secondary rays restart from the hit triangle into the tet the primary ray
arrived from (Sec. 6 of the paper: scattered rays start from a tet adjacent
to the hit face, so the same face is not intersected again).  Two kinds:

* diffuse bounce: one cosine-weighted direction per hit, unbounded t_max;
* ambient occlusion: K cosine-weighted directions per hit, t_max = 0.05.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of a stream seeded with s is mix64(s + (i+1)*gamma).
Uniform u = (x >> 40) * 2^-24 (exact in float32 and float64).  Draw index of
ray k of hit r, coordinate j in {0, 1}: 2*(r*K + k) + j.

Direction: phi = 2*pi*u0, s = sqrt(u1), local = (s cos phi, s sin phi,
sqrt(1 - u1)), mapped with the branchless orthonormal basis of Duff et al.,
"Building an Orthonormal Basis, Revisited" (JCGT 2017) around the unit
normal of the triangle's own plane ((v1-v0) x (v2-v0)), flipped to the
arrival side.  Origin: (1-b1-b2) v0 + b1 v1 + b2 v2.  All in float64, one
rounding to float32 at the end.
"""
from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MUL2)
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, counter: np.ndarray) -> np.ndarray:
    """u in [0,1), a multiple of 2^-24, for each counter value."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & M64) + (c + np.uint64(1)) * np.uint64(GAMMA)
    return (mix64(z) >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))


def duff_onb(n: np.ndarray):
    """Orthonormal b1, b2 completing unit normals n [N,3] (Duff et al. 2017)."""
    sign = np.where(n[:, 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1.0 + sign * n[:, 0] * n[:, 0] * a, sign * b, -sign * n[:, 0]], axis=1)
    b2 = np.stack([b, sign + n[:, 1] * n[:, 1] * a, -n[:, 1]], axis=1)
    return b1, b2


def secondary_rays(points, tris, hit_tri, hit_b1, hit_b2, hit_side, seed: int, per_hit: int,
                   tmax: float, ray_ids=None):
    """Rays for every hit (hit_tri >= 0), `per_hit` each.

    hit_side: 0 when the primary ray arrived from the + side of its triangle
    (the side its normal (v1-v0)x(v2-v0) points to), 1 from the - side.
    Returns o, d (float32 [M,3]), tmax (float32 [M]), entry = 2*tri + side
    (int32 [M]) and src (int64 [M], the primary ray index of each).
    `ray_ids` gives the counter index of each hit (defaults to its position).
    """
    P = np.asarray(points, dtype=np.float64)
    tris = np.asarray(tris)
    hit_tri = np.asarray(hit_tri)
    sel = np.nonzero(hit_tri >= 0)[0]
    rid = sel if ray_ids is None else np.asarray(ray_ids)[sel]
    c = hit_tri[sel].astype(np.int64)
    v0, v1, v2 = P[tris[c, 0]], P[tris[c, 1]], P[tris[c, 2]]
    b1 = np.asarray(hit_b1, dtype=np.float64)[sel]
    b2 = np.asarray(hit_b2, dtype=np.float64)[sel]
    x = (1.0 - b1 - b2)[:, None] * v0 + b1[:, None] * v1 + b2[:, None] * v2
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    side = np.asarray(hit_side)[sel].astype(np.int64)
    nrm = np.where((side == 1)[:, None], -nrm, nrm)
    e1, e2 = duff_onb(nrm)
    K = per_hit
    o_list, d_list, entry_list, src_list = [], [], [], []
    for k in range(K):
        cnt = 2 * (rid.astype(np.uint64) * np.uint64(K) + np.uint64(k))
        u0 = uniform(seed, cnt)
        u1 = uniform(seed, cnt + np.uint64(1))
        phi = 2.0 * math.pi * u0
        s = np.sqrt(u1)
        lz = np.sqrt(np.maximum(0.0, 1.0 - u1))
        dirs = (s * np.cos(phi))[:, None] * e1 + (s * np.sin(phi))[:, None] * e2 + lz[:, None] * nrm
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        o_list.append(x)
        d_list.append(dirs)
        entry_list.append(2 * c + side)
        src_list.append(sel)
    # interleave so that the K rays of one hit are consecutive
    o = np.stack(o_list, axis=1).reshape(-1, 3).astype(np.float32)
    d = np.stack(d_list, axis=1).reshape(-1, 3).astype(np.float32)
    entry = np.stack(entry_list, axis=1).reshape(-1).astype(np.int32)
    src = np.stack(src_list, axis=1).reshape(-1).astype(np.int64)
    tm = np.full(len(o), tmax, dtype=np.float32)
    return o, d, tm, entry, src


def hit_side(ctet: np.ndarray, hit_tri: np.ndarray, hit_tet: np.ndarray) -> np.ndarray:
    """Side (0 = +, 1 = -) of each hit triangle on which its terminating tet lies."""
    side = np.zeros(len(hit_tri), dtype=np.int32)
    ok = hit_tri >= 0
    side[ok] = np.where(ctet[hit_tri[ok], 0] == hit_tet[ok], 0, 1)
    return side


def arrival_side(points, tris, hit_tri, d) -> np.ndarray:
    """Side (0 = +, 1 = -) from which each ray of direction d arrives at its
    hit triangle, from the geometry alone: a ray travelling against the
    normal (v1-v0)x(v2-v0) comes from the side the normal points to.  Equals
    hit_side for every hit that is not tangent to its triangle; needs no tets."""
    P = np.asarray(points, dtype=np.float64)
    tris = np.asarray(tris)
    hit_tri = np.asarray(hit_tri)
    side = np.zeros(len(hit_tri), dtype=np.int32)
    ok = hit_tri >= 0
    c = hit_tri[ok].astype(np.int64)
    v0, v1, v2 = P[tris[c, 0]], P[tris[c, 1]], P[tris[c, 2]]
    nd = (np.cross(v1 - v0, v2 - v0) * np.asarray(d, dtype=np.float64)[ok]).sum(1)
    side[ok] = np.where(nd < 0.0, 0, 1)
    return side


def _hit_points(points, tris, hit_tri, hit_b1, hit_b2):
    """Selected hit rows, triangle ids, hit points, first vertices and unnormalised normals (FP64)."""
    P = np.asarray(points, dtype=np.float64)
    tris = np.asarray(tris)
    hit_tri = np.asarray(hit_tri)
    sel = np.nonzero(hit_tri >= 0)[0]
    c = hit_tri[sel].astype(np.int64)
    v0, v1, v2 = P[tris[c, 0]], P[tris[c, 1]], P[tris[c, 2]]
    b1 = np.asarray(hit_b1, dtype=np.float64)[sel]
    b2 = np.asarray(hit_b2, dtype=np.float64)[sel]
    x = (1.0 - b1 - b2)[:, None] * v0 + b1[:, None] * v1 + b2[:, None] * v2
    nrm = np.cross(v1 - v0, v2 - v0)
    return sel, c, x, v0, nrm


def shadow_rays(points, tris, hit_tri, hit_b1, hit_b2, light):
    """Shadow rays toward a point light (Sec. 6), one per hit (hit_tri >= 0).

    From the hit point x toward L: d = (L - x)/|L - x|, tmax = |L - x|,
    restarted from the hit triangle into the side that faces L (0, the +
    side, when n . (L - v0) >= 0, n = (v1-v0) x (v2-v0); else 1).  Returns
    o, d (float32 [M,3]), tmax (float32 [M]), entry = 2*tri + side (int32)
    and src (int64, the hit index of each ray).
    """
    sel, c, x, v0, nrm = _hit_points(points, tris, hit_tri, hit_b1, hit_b2)
    L = np.asarray(light, dtype=np.float64).reshape(1, 3)
    side = np.where(np.einsum("ij,ij->i", nrm, L - v0) >= 0.0, 0, 1)
    v = L - x
    ln = np.linalg.norm(v, axis=1)
    d = v / ln[:, None]
    return (x.astype(np.float32), d.astype(np.float32), ln.astype(np.float32),
            (2 * c + side).astype(np.int32), sel.astype(np.int64))


def specular_rays(points, tris, hit_tri, hit_b1, hit_b2, hit_side, d_in, kind: str, ior: float,
                  tmax: float):
    """Reflection or refraction rays (Sec. 6), one per hit (hit_tri >= 0).

    w = d_in / |d_in| (the incoming ray of each hit), n_a = the unit normal
    turned toward the arrival side (hit_side 0: +, 1: -), c = max(0, -w.n_a).
    Mirror direction r = w + 2 c n_a (Snell's law of reflection), restarted
    on the arrival side.  Refraction (Snell's law, vector form): with eta the
    ratio of refractive indices arrival side / far side (ior from the - side,
    1/ior from the + side; ior = index of the - side over the + side) and
    k = 1 - eta^2 (1 - c^2), the transmitted direction is
    eta w + (eta c - sqrt(k)) n_a, restarted on the far side; k < 0 is total
    internal reflection and gives the mirror direction.  Directions are
    normalised; float64 throughout, one rounding to float32.  Returns o, d,
    tmax, entry = 2*tri + side, src as shadow_rays, and k (float64).
    """
    sel, c, x, v0, nrm = _hit_points(points, tris, hit_tri, hit_b1, hit_b2)
    side = np.asarray(hit_side)[sel].astype(np.int64)
    n = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    na = np.where((side == 1)[:, None], -n, n)
    w = np.asarray(d_in, dtype=np.float64)[sel]
    w = w / np.linalg.norm(w, axis=1, keepdims=True)
    cs = np.maximum(0.0, -np.einsum("ij,ij->i", w, na))
    eta = np.where(side == 1, float(ior), 1.0 / float(ior))
    k = 1.0 - eta * eta * (1.0 - cs * cs)
    refl = w + (2.0 * cs)[:, None] * na
    if kind == "refract":
        ok = k >= 0.0
        tr = eta[:, None] * w + (eta * cs - np.sqrt(np.maximum(k, 0.0)))[:, None] * na
        d = np.where(ok[:, None], tr, refl)
        out_side = np.where(ok, 1 - side, side)
    elif kind == "reflect":
        d = refl
        out_side = side
    else:
        raise ValueError(kind)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    tm = np.full(len(sel), tmax, dtype=np.float32)
    return (x.astype(np.float32), d.astype(np.float32), tm, (2 * c + out_side).astype(np.int32),
            sel.astype(np.int64), k)
