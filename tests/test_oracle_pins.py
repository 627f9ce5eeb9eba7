"""Pins of the FP64 oracle to things other than itself.

* brute force over every constrained triangle (walk == nearest triangle),
* closed forms: a constrained plane z = z0 (exact t, triangle id and
  barycentrics) and a voxelised sphere (t bracketed by the spheres of radius
  r -/+ delta),
* mesh invariants (orientation, neighbour symmetry, boundary face count),
* restart rays through the hit face (walk with the entry face excluded ==
  brute force without the source triangle),
* point location (the located tet holds the point),
* the secondary-ray generator (published SplitMix64 outputs, hemisphere and
  cosine-law moments).
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from oracle.secondary import arrival_side, mix64, secondary_rays, hit_side, uniform, GAMMA, M64

ROOT_GOLDEN = __file__.rsplit("/", 1)[0] + "/golden"


def edge_margin(points, tris, tri, b1, b2):
    """Distance-like margin of a hit from its triangle's edges (min barycentric x edge length)."""
    P = np.asarray(points, np.float64)
    v0, v1, v2 = P[tris[tri, 0]], P[tris[tri, 1]], P[tris[tri, 2]]
    size = np.maximum.reduce([np.linalg.norm(v1 - v0, axis=1), np.linalg.norm(v2 - v1, axis=1),
                              np.linalg.norm(v0 - v2, axis=1)])
    return np.minimum.reduce([b1, b2, 1.0 - b1 - b2]) * size


def random_scene(n, seed, frac=0.3, jitter=0.2):
    pts, tets = sg.freudenthal_grid(n, jitter, seed)
    inside = np.random.default_rng(seed).random((n, n, n)) < frac
    tris = sg.constrained_faces(n, inside)
    return pts, tets, tris


def random_rays(m, count, seed):
    g = np.random.default_rng(seed)
    q = g.uniform(0.02, 0.98, size=(count, 3)).astype(np.float32)
    start, mb = m.locate(q)
    d = g.normal(size=(count, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    keep = mb > 1e-9
    return q[keep], d[keep], start[keep]


def compare_walk_brute(points, tris, w, b, tol=1e-9):
    same = w["tri"] == b["tri"]
    bad = ~same
    # a mismatch is excused only when the true (brute-force) hit lies on an edge
    hit = bad & (b["tri"] >= 0)
    if hit.any():
        marg = edge_margin(points, tris, b["tri"][hit], b["b1"][hit], b["b2"][hit])
        assert (marg < tol).all(), f"walk/brute mismatch away from edges: {marg.min()}"
    assert not (bad & (b["tri"] < 0)).any(), "walk reports a hit where nothing is hit"
    both = same & (w["tri"] >= 0)
    np.testing.assert_allclose(w["t"][both], b["t"][both], rtol=1e-12, atol=0)
    return same.mean()


def test_invariants_tiny():
    s = sg.make_config("tiny")
    m = oracle.OracleMesh(s.points, s.tets, s.tris)
    assert m.count_nonpositive() == 0
    assert m.count_asymmetric() == 0
    assert m.count_boundary() == 12 * s.n * s.n            # 6 cube faces x n^2 squares x 2
    nbr, fc, ctet = m.arrays()
    interior = (nbr >= 0).sum()
    assert interior == 4 * s.n_tets - 12 * s.n * s.n
    assert (ctet >= 0).all()                                # every triangle has a tet on both sides
    assert ((fc >= 0).sum()) == 2 * s.n_tris


def test_asymmetry_checker_counts_planted_links():
    """The neighbour-symmetry checker is a detector, not a constant: swap the
    links of one interior tet across two of its faces.  Its own two links
    now name a neighbour that points back through a face with other
    vertices (caught by the vertex comparison), and its two former
    neighbours point to a tet that no longer points back (caught by the
    back-link test): exactly four defects."""
    s = sg.make_config("tiny")
    m = oracle.OracleMesh(s.points, s.tets, s.tris)
    assert m.count_asymmetric() == 0
    nbr, _, _ = m.arrays()
    t = int(np.nonzero((nbr >= 0).all(axis=1))[0][0])
    k1, k2 = 0, 1
    u1, u2 = int(nbr[t, k1]), int(nbr[t, k2])
    ku1 = int(np.nonzero(nbr[u1] == t)[0][0])
    ku2 = int(np.nonzero(nbr[u2] == t)[0][0])
    m.relink(t, k1, u2, ku2)
    m.relink(t, k2, u1, ku1)
    assert m.count_asymmetric() == 4
    # a one-sided link to the boundary: its old neighbour no longer sees a link back
    m2 = oracle.OracleMesh(s.points, s.tets, s.tris)
    m2.relink(t, k1, -1, -1)
    assert m2.count_asymmetric() == 1


def test_rejects_bad_meshes():
    pts, tets = sg.freudenthal_grid(2, 0.0, 1)
    tris = np.array([[0, 1, 2]], np.int32)                  # not a face of the Kuhn split
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(pts, tets, tris)
    bad = tets.copy(); bad[0, 0] = 10_000
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(pts, bad, np.zeros((0, 3), np.int32))
    dup = np.concatenate([tets, tets[:1]])                  # a face shared by three tets
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(pts, dup, np.zeros((0, 3), np.int32))
    flipped = tets.copy(); flipped[0, [2, 3]] = flipped[0, [3, 2]]
    m = oracle.OracleMesh(pts, flipped, np.zeros((0, 3), np.int32))
    assert m.count_nonpositive() == 1


def test_walk_equals_bruteforce_tiny_camera():
    s = sg.make_config("tiny")
    m = oracle.OracleMesh(s.points, s.tets, s.tris)
    tet, mb = m.locate(np.array([s.camera.eye], np.float32))
    assert mb[0] > 1e-6
    o, d = sg.camera_rays(s.camera)
    w = m.trace(o, d, np.inf, tet[0])
    b = m.bruteforce(o, d, np.inf)
    assert (w["flags"] == 0).all()
    assert compare_walk_brute(s.points, s.tris, w, b) == 1.0


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_walk_equals_bruteforce_random_meshes(seed):
    n = 3 + seed % 3
    pts, tets, tris = random_scene(n, seed)
    m = oracle.OracleMesh(pts, tets, tris)
    assert m.count_nonpositive() == 0 and m.count_asymmetric() == 0
    q, d, start = random_rays(m, 1500, seed)
    w = m.trace(q, d, np.inf, start)
    b = m.bruteforce(q, d, np.inf)
    assert ((w["flags"] & ~oracle.FLAG_TIE) == 0).all()
    assert compare_walk_brute(pts, tris, w, b) > 0.999
    # finite t_max: hits beyond it become misses in both
    tm = np.random.default_rng(seed).uniform(0.0, 0.6, size=len(q)).astype(np.float32)
    w2 = m.trace(q, d, tm, start)
    b2 = m.bruteforce(q, d, tm)
    compare_walk_brute(pts, tris, w2, b2)
    assert (w2["tri"] >= 0).sum() < (w["tri"] >= 0).sum()
    # a ray cut short by t_max stops in the tet that holds its end point
    end = q.astype(np.float64) + tm[:, None].astype(np.float64) * d.astype(np.float64)
    inside = (end > 1e-6).all(1) & (end < 1 - 1e-6).all(1)
    cut = (w2["tri"] < 0) & inside & (w["t"] > tm)
    assert cut.sum() > 50
    for r in np.nonzero(cut)[0]:
        assert m.tet_bary(w2["tet"][r], end[r]).min() > -1e-9


def test_walk_t_increases():
    s = sg.make_config("medium")
    m = oracle.OracleMesh(s.points, s.tets, s.tris)
    tet, _ = m.locate(np.array([s.camera.eye], np.float32))
    o, d = sg.camera_rays(s.camera)
    sel = np.random.default_rng(0).choice(len(o), 4000, replace=False)
    w = m.trace(o[sel], d[sel], np.inf, tet[0])
    assert (w["flags"] & ~oracle.FLAG_TIE == 0).all()   # exit t never decreases, no degenerate tet
    assert (w["flags"] & oracle.FLAG_TIE).astype(bool).mean() < 1e-3   # edge/vertex ties are rare
    assert w["steps"].max() > 50            # long walks through many tets


def slab_expected(n, layer, o, d):
    """Exact hit of the plane z = z0 tiled by the Kuhn face split (grid lines at float32(i*h))."""
    grid = (np.arange(n + 1) * (1.0 / n)).astype(np.float32).astype(np.float64)
    z0 = grid[layer]
    t = (z0 - o[:, 2].astype(np.float64)) / d[:, 2].astype(np.float64)
    x = o.astype(np.float64) + t[:, None] * d.astype(np.float64)
    i = np.searchsorted(grid, x[:, 0], side="right") - 1
    j = np.searchsorted(grid, x[:, 1], side="right") - 1
    fx = (x[:, 0] - grid[i]) / (grid[i + 1] - grid[i])
    fy = (x[:, 1] - grid[j]) / (grid[j + 1] - grid[j])
    half = (fy > fx).astype(np.int64)
    tri = 2 * (i + n * j) + half
    b1 = np.where(half == 0, fx - fy, fx)
    b2 = np.where(half == 0, fy, fy - fx)
    return tri, t, b1, b2


@pytest.mark.parametrize("direction", [+1, -1])
def test_closed_form_plane(direction):
    n, layer = 6, 2
    pts, tets = sg.freudenthal_grid(n, 0.0, 5)
    tris = sg.constrained_faces(n, sg.slab_cells(n, layer))
    assert len(tris) == 2 * n * n
    m = oracle.OracleMesh(pts, tets, tris)
    g = np.random.default_rng(7)
    cnt = 3000
    z = g.uniform(0.02, layer / n - 0.05, cnt) if direction > 0 else g.uniform(layer / n + 0.05, 0.98, cnt)
    o = np.stack([g.uniform(0.2, 0.8, cnt), g.uniform(0.2, 0.8, cnt), z], axis=1).astype(np.float32)
    d = np.stack([g.uniform(-0.3, 0.3, cnt), g.uniform(-0.3, 0.3, cnt),
                  np.full(cnt, float(direction))], axis=1)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    start, mb = m.locate(o)
    keep = mb > 1e-9
    o, d, start = o[keep], d[keep], start[keep]
    tri, t, b1, b2 = slab_expected(n, layer, o, d)
    inside = (b1 > 1e-9) & (b2 > 1e-9) & (1 - b1 - b2 > 1e-9)
    for res in (m.trace(o, d, np.inf, start), m.bruteforce(o, d, np.inf)):
        assert (res["tri"][inside] == tri[inside]).all()
        np.testing.assert_allclose(res["t"], t, rtol=1e-12)
        np.testing.assert_allclose(res["b1"][inside], b1[inside], atol=1e-10)
        np.testing.assert_allclose(res["b2"][inside], b2[inside], atol=1e-10)


def test_closed_form_sphere():
    n, j = 24, 0.15
    centre, r = np.array([0.5, 0.5, 0.55]), 0.3
    pts, tets = sg.freudenthal_grid(n, j, 21)
    tris = sg.constrained_faces(n, sg.inside_cells(n, centre[None], np.array([r])))
    m = oracle.OracleMesh(pts, tets, tris)
    eye = np.array([[0.5, 0.47, 0.08]], np.float32)
    start, mb = m.locate(eye)
    g = np.random.default_rng(3)
    cnt = 4000
    target = centre + g.uniform(-0.45, 0.45, size=(cnt, 3))
    d = target - eye.astype(np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    o = np.repeat(eye, cnt, axis=0)
    w = m.trace(o, d, np.inf, start[0])
    h = 1.0 / n
    delta = math.sqrt(3.0) * (0.5 + j) * h
    oc = o.astype(np.float64) - centre
    dd = d.astype(np.float64)
    a = (dd * dd).sum(1)
    bq = (oc * dd).sum(1)
    imp = np.sqrt(np.maximum(0.0, (oc * oc).sum(1) - bq * bq / a))   # impact parameter

    def t_sphere(rad):
        disc = bq * bq - a * ((oc * oc).sum(1) - rad * rad)
        return (-bq - np.sqrt(np.maximum(disc, 0.0))) / a

    must_hit = imp < r - delta - 1e-9
    must_miss = imp > r + delta + 1e-9
    assert must_hit.sum() > 500 and must_miss.sum() > 500
    assert (w["tri"][must_hit] >= 0).all()
    assert (w["tri"][must_miss] < 0).all()
    tv = w["t"][must_hit]
    assert (tv >= t_sphere(r + delta)[must_hit] - 1e-12).all()
    assert (tv <= t_sphere(r - delta)[must_hit] + 1e-12).all()


def test_restart_rays_equal_bruteforce():
    pts, tets, tris = random_scene(5, 31, frac=0.35)
    m = oracle.OracleMesh(pts, tets, tris)
    q, d, start = random_rays(m, 2000, 31)
    w = m.trace(q, d, np.inf, start)
    nbr, fc, ctet = m.arrays()
    side = hit_side(ctet, w["tri"], w["tet"])
    # the terminating tet really lies on that face
    hit = w["tri"] >= 0
    assert (fc[w["tet"][hit]] == w["tri"][hit][:, None]).any(axis=1).all()
    o2, d2, tm2, entry, src = secondary_rays(pts, tris, w["tri"], w["b1"], w["b2"], side,
                                             seed=99, per_hit=2, tmax=np.inf)
    assert len(o2) == 2 * hit.sum()
    w2 = m.trace(o2, d2, tm2, -1, entry)
    assert (w2["flags"] & oracle.FLAG_BAD_START == 0).all()
    b2 = m.bruteforce(o2, d2, tm2, exclude=entry >> 1)
    assert compare_walk_brute(pts, tris, w2, b2, tol=1e-7) > 0.995
    # AO: bounded rays
    o3, d3, tm3, entry3, _ = secondary_rays(pts, tris, w["tri"], w["b1"], w["b2"], side,
                                            seed=5, per_hit=8, tmax=0.05)
    w3 = m.trace(o3, d3, tm3, -1, entry3)
    b3 = m.bruteforce(o3, d3, tm3, exclude=entry3 >> 1)
    compare_walk_brute(pts, tris, w3, b3, tol=1e-7)
    assert (w3["t"][w3["tri"] >= 0] <= 0.05).all()


def test_triangle_set_bruteforce_and_arrival_side():
    """The tet-free triangle set (for scenes too large for the adjacency
    build) finds the walk's hits, and the side a ray arrives from, taken from
    the geometry alone, is the side of the tet the walk ends in."""
    pts, tets, tris = random_scene(5, 57, frac=0.35)
    m = oracle.OracleMesh(pts, tets, tris)
    ts = oracle.OracleTriangles(pts, tris)
    q, d, start = random_rays(m, 3000, 57)
    w = m.trace(q, d, np.inf, start)
    b = ts.bruteforce(q, d, np.inf)
    assert compare_walk_brute(pts, tris, w, b, tol=1e-7) > 0.995
    hit = w["tri"] >= 0
    assert hit.sum() > 1000
    _, _, ctet = m.arrays()
    np.testing.assert_array_equal(arrival_side(pts, tris, w["tri"], d), hit_side(ctet, w["tri"], w["tet"]))
    with pytest.raises(oracle.OracleError):
        ts.trace(q, d, np.inf, start)


def test_locate_contains_point():
    pts, tets, tris = random_scene(4, 41)
    m = oracle.OracleMesh(pts, tets, tris)
    q = np.random.default_rng(4).uniform(0, 1, size=(300, 3)).astype(np.float32)
    tet, mb = m.locate(q)
    assert (mb > -1e-12).all()
    for i in range(0, 300, 37):
        w = m.tet_bary(tet[i], q[i].astype(np.float64))
        assert abs(w.sum() - 1.0) < 1e-12 and w.min() > -1e-12


def test_splitmix64_published_outputs():
    vals = [int(line, 16) for line in open(f"{ROOT_GOLDEN}/splitmix64_seed0.txt")
            if line.strip() and not line.startswith("#")]
    got, z = [], 0
    for _ in range(3):
        z = (z + GAMMA) & M64
        got.append(int(mix64(np.array([z], np.uint64))[0]))
    assert got == vals
    u = uniform(0, np.arange(3, dtype=np.uint64))
    assert np.allclose(u, [(v >> 40) / 2 ** 24 for v in vals])


def test_secondary_directions_cosine_law():
    s = sg.make_config("tiny")
    m = oracle.OracleMesh(s.points, s.tets, s.tris)
    tet, _ = m.locate(np.array([s.camera.eye], np.float32))
    o, d = sg.camera_rays(s.camera)
    w = m.trace(o, d, np.inf, tet[0])
    _, _, ctet = m.arrays()
    side = hit_side(ctet, w["tri"], w["tet"])
    o2, d2, _, entry, src = secondary_rays(s.points, s.tris, w["tri"], w["b1"], w["b2"], side,
                                           seed=1, per_hit=16, tmax=np.inf)
    P = s.points.astype(np.float64)
    c = entry >> 1
    nrm = np.cross(P[s.tris[c, 1]] - P[s.tris[c, 0]], P[s.tris[c, 2]] - P[s.tris[c, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm[(entry & 1) == 1] *= -1
    cos = (d2.astype(np.float64) * nrm).sum(1)
    assert (cos > 0).all()                                        # back into the arrival side
    assert (np.einsum("ij,ij->i", d[src].astype(np.float64), nrm) < 0).all()
    assert abs(cos.mean() - 2.0 / 3.0) < 0.01                     # E[cos] = 2/3 under the cosine law
    assert abs((cos ** 2).mean() - 0.5) < 0.01                    # E[cos^2] = 1/2
    np.testing.assert_allclose(np.linalg.norm(d2, axis=1), 1.0, atol=1e-6)
