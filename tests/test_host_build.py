"""Host-side checks of the CUDA library (no GPU needed): symbols, packing,
Hilbert order and build errors.  The packed records are checked against the
oracle's independent adjacency through the xor identities of Sec. 3.
"""
import os
import re

import numpy as np
import pytest

import oracle
import scenegen as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAG = np.uint32(0x80000000)
BOUNDARY = np.uint32(0xFFFFFFFF)


@pytest.fixture(scope="module")
def tmx():
    from paper_2103_02309_gb300 import build
    build.build()
    from paper_2103_02309_gb300 import tetmesh
    return tetmesh


def header_functions():
    src = open(os.path.join(ROOT, "include", "tetmesh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(tmx):
    from paper_2103_02309_gb300 import _native as N
    declared = header_functions()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(N.lib, name), f"{name} declared in tetmesh.h but not exported"
    assert set(N.EXPORTED) <= set(declared)


def test_bench_probe_is_a_library_of_its_own(tmx):
    """The benchmark's read-bandwidth probe is outside the C ABI: its own
    library exports it, the traversal library does not."""
    import ctypes
    from paper_2103_02309_gb300 import _native as N
    from paper_2103_02309_gb300 import build as libbuild
    assert not hasattr(N.lib, "tm_read_probe") and not hasattr(N.lib, "tm_bench_read_probe")
    probe = ctypes.CDLL(libbuild.PROBE_LIB)
    assert hasattr(probe, "tm_bench_read_probe")


def expected_raw_neighbours(om, tinv):
    """Neighbour field values the packing must produce, per (input tet, local face)."""
    nbr, fc, _ = om.arrays()
    raw = np.where(nbr >= 0, tinv[np.maximum(nbr, 0)].astype(np.int64), BOUNDARY.astype(np.int64))
    raw = np.where(fc >= 0, (FLAG.astype(np.int64) | fc.astype(np.int64)), raw)
    return raw.astype(np.int64) & 0xFFFFFFFF


@pytest.mark.parametrize("order", ["hilbert", "input"])
@pytest.mark.parametrize("name,n", [("tiny", None), ("medium", 16)])
def test_packing_matches_oracle_adjacency(tmx, name, n, order):
    s = sg.make_config(name, n_override=n)
    m = tmx.Mesh(s.points, s.tets, s.tris, order=order, upload=False)
    e = m.export()
    tperm, pperm = e["tet_perm"], e["point_perm"]
    assert np.array_equal(np.sort(tperm), np.arange(s.n_tets))
    assert np.array_equal(np.sort(pperm), np.arange(s.n_points))
    if order == "input":
        assert np.array_equal(tperm, np.arange(s.n_tets))
    tinv = np.empty_like(tperm); tinv[tperm] = np.arange(len(tperm))
    pinv = np.empty_like(pperm); pinv[pperm] = np.arange(len(pperm))
    # points are the input points, renumbered
    assert np.array_equal(e["points"][:, :3], s.points[pperm])
    assert (e["points"][:, 3] == 0).all()
    # cold records: input vertex order (positive orientation), N_k across V_k
    cold = e["cold"]
    assert np.array_equal(cold[:, :4], pinv[s.tets[tperm]])
    om = oracle.OracleMesh(s.points, s.tets, s.tris)
    raw = expected_raw_neighbours(om, tinv)
    assert np.array_equal(cold[:, 4:].astype(np.int64) & 0xFFFFFFFF, raw[tperm])
    # Tet16: VX = V0^V1^V2^V3 ; NX_j = N_j ^ N_3 with neighbours sorted by vertex id
    V = cold[:, :4].astype(np.int64)
    Nb = cold[:, 4:].astype(np.int64) & 0xFFFFFFFF
    order_ = np.argsort(V, axis=1, kind="stable")
    Vs = np.take_along_axis(V, order_, 1)
    Ns = np.take_along_axis(Nb, order_, 1)
    t16 = e["tet16"].astype(np.int64) & 0xFFFFFFFF
    assert np.array_equal(t16[:, 0], Vs[:, 0] ^ Vs[:, 1] ^ Vs[:, 2] ^ Vs[:, 3])
    for j in range(3):
        assert np.array_equal(t16[:, 1 + j], Ns[:, j] ^ Ns[:, 3])
    # Decoding (Alg. 7): from the neighbour at any rank, every other one is recovered
    NXe = np.concatenate([t16[:, 1:], np.zeros((len(t16), 1), np.int64)], axis=1)
    for ra in range(4):
        n3 = Ns[:, ra] ^ NXe[:, ra]
        for rb in range(4):
            assert np.array_equal(n3 ^ NXe[:, rb], Ns[:, rb])
    # the fourth vertex from three (Sec. 3: V3 = V0 ^ V1 ^ V2 ^ VX)
    assert np.array_equal(Vs[:, 0] ^ Vs[:, 1] ^ Vs[:, 2] ^ t16[:, 0], Vs[:, 3])
    # constrained-face table: tri, tet on the + side, tet on the - side, own vertex order
    _, _, ctet = om.arrays()
    cf = e["cface"]
    assert np.array_equal(cf[:, 0], np.arange(s.n_tris))
    assert np.array_equal(cf[:, 1], np.where(ctet[:, 0] >= 0, tinv[np.maximum(ctet[:, 0], 0)], -1))
    assert np.array_equal(cf[:, 2], np.where(ctet[:, 1] >= 0, tinv[np.maximum(ctet[:, 1], 0)], -1))
    assert np.array_equal(cf[:, 4:7], pinv[s.tris])
    # id maps
    assert np.array_equal(m.map_ids(tmx.IDS_TET, tmx.TO_INPUT, np.arange(s.n_tets)), tperm)
    assert np.array_equal(m.map_ids(tmx.IDS_TET, tmx.TO_INTERNAL, tperm), np.arange(s.n_tets))
    assert np.array_equal(m.map_ids(tmx.IDS_POINT, tmx.TO_INTERNAL, [-5, s.n_points]), [-1, -1])
    info = m.info
    assert info.n_tets == s.n_tets and info.on_device == 0 and abs(info.extent - 1.0) < 1e-6


def test_hilbert_order_improves_locality(tmx):
    """A compact block of cells spans fewer 4 KB pages of Tet16 records in Hilbert order."""
    n = 32
    s = sg.make_config("medium", n_override=n)
    rng = np.random.default_rng(0)
    corners = rng.integers(0, n - 8, size=(12, 3))
    pages = {}
    for order in ("hilbert", "input"):
        e = tmx.Mesh(s.points, s.tets, s.tris, order=order, upload=False).export()
        tinv = np.empty_like(e["tet_perm"]); tinv[e["tet_perm"]] = np.arange(len(tinv))
        cnt = []
        for a, b, c in corners:
            k, j, i = np.meshgrid(np.arange(c, c + 8), np.arange(b, b + 8), np.arange(a, a + 8),
                                  indexing="ij")
            cube = (i + n * (j + n * k)).ravel()
            tets = (6 * cube[:, None] + np.arange(6)).ravel()
            cnt.append(len(np.unique(tinv[tets] // 256)))
        pages[order] = np.mean(cnt)
    assert pages["hilbert"] < 0.8 * pages["input"], pages


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_curve_bijective_and_adjacent(tmx, bits):
    side = 1 << bits
    g = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij"),
                 axis=-1).reshape(-1, 3).astype(np.uint32)
    k = tmx.hilbert_keys(g, bits)
    assert np.array_equal(np.sort(k), np.arange(side ** 3, dtype=np.uint64))
    path = g[np.argsort(k)].astype(np.int64)
    step = np.abs(np.diff(path, axis=0)).sum(axis=1)
    assert (step == 1).all()                 # consecutive cells share a face


def test_build_errors(tmx):
    from paper_2103_02309_gb300 import _native as N
    pts, tets = sg.freudenthal_grid(3, 0.1, 7)
    tris = sg.constrained_faces(3, sg.slab_cells(3, 1))
    tmx.Mesh(pts, tets, tris, upload=False)                        # valid
    cases = {
        2: (pts, np.where(np.arange(tets.size).reshape(tets.shape) == 5, 10_000, tets), tris),
        3: (pts, tets[:, [0, 1, 3, 2]], tris),                      # every tet flipped
        4: (pts, np.concatenate([tets, tets[:1]]), tris),           # a face shared by three tets
        5: (pts, tets, np.array([[0, 1, 2]], np.int32)),            # not a face of any tet
        6: (pts, tets, np.concatenate([tris, tris[:1]])),           # two triangles on one face
    }
    for status, (p, t, c) in cases.items():
        with pytest.raises(N.TetmeshError) as ei:
            tmx.Mesh(p, t, c, upload=False)
        assert ei.value.status == status, (status, str(ei.value))
    # ray and hit buffers must be 32-byte aligned: refused before the device is touched
    m0 = tmx.Mesh(pts, tets, tris, upload=False)
    lib = N.lib
    assert lib.tm_trace(m0._h, 16, 1, None, 64, None, None) == 1          # TM_ERR_ARG
    assert lib.tm_trace(m0._h, 64, 1, None, 48, None, None) == 1
    assert lib.tm_trace(m0._h, 64, 1, None, 96, None, None) != 1         # aligned: TM_ERR_NO_DEVICE
    # a flipped mesh is accepted when asked to fix orientation, with positive tets
    m = tmx.Mesh(pts, tets[:, [0, 1, 3, 2]], tris, upload=False, fix_orientation=True)
    cold = m.export()["cold"]
    P = m.export()["points"][:, :3].astype(np.float64)
    a, b, c, d = (P[cold[:, k]] for k in range(4))
    assert (np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) > 0).all()


def test_tet20_records(tmx):
    """Tet20 (Sec. 3): VX and the four neighbours sorted by the ids of the vertices they sit across."""
    s = sg.make_config("tiny")
    m = tmx.Mesh(s.points, s.tets, s.tris, upload=False, tet20=True)
    e = m.export()
    t20 = m.export_tet20()
    V = e["cold"][:, :4].astype(np.int64)
    Nb = e["cold"][:, 4:].astype(np.int64) & 0xFFFFFFFF
    order = np.argsort(V, axis=1, kind="stable")
    Ns = np.take_along_axis(Nb, order, 1)
    assert np.array_equal(t20["vxn"][:, 0], e["tet16"][:, 0])
    assert np.array_equal(t20["vxn"][:, 1:].astype(np.int64) & 0xFFFFFFFF, Ns[:, :3])
    assert np.array_equal(t20["n3"].astype(np.int64) & 0xFFFFFFFF, Ns[:, 3])
    assert np.array_equal(t20["aos"][:, :4], t20["vxn"]) and np.array_equal(t20["aos"][:, 4], t20["n3"])
    from paper_2103_02309_gb300 import _native as N
    with pytest.raises(N.TetmeshError):
        tmx.Mesh(s.points, s.tets, s.tris, upload=False).export_tet20()


def test_hilbert_regions_order(tmx):
    """Regions (Sec. 5): tets enclosed by the same constrained faces are stored
    together, regions in order of their first Hilbert key, Hilbert order inside.

    Reference regions come from the scene's cell labels: on the Kuhn grid two
    cells share a non-constrained face exactly when both are inside or both
    outside, so the regions are the face-connected components of the inside
    cells and of the outside cells."""
    ndimage = pytest.importorskip("scipy.ndimage")
    n = 16
    s = sg.make_config("medium", n_override=n)
    m = tmx.Mesh(s.points, s.tets, s.tris, order="hilbert_regions", upload=False)
    e = m.export()
    lab_in, k_in = ndimage.label(s.inside)
    lab_out, k_out = ndimage.label(~s.inside)
    cell_region = np.where(s.inside, lab_in - 1, k_in + lab_out - 1).ravel()  # [k, j, i] order
    tet_region = np.repeat(cell_region, 6)                                   # tet = 6*cube + p
    assert m.info.n_regions == k_in + k_out
    internal_region = tet_region[e["tet_perm"]]
    # each region occupies one contiguous run of internal ids
    changes = np.count_nonzero(np.diff(internal_region)) + 1
    assert changes == k_in + k_out
    # Hilbert keys of the centroids (2^21 grid over the unit cube) rise inside a region,
    # and regions follow the order of their smallest key
    c = s.points.astype(np.float64)[s.tets].mean(axis=1)[e["tet_perm"]]
    q = np.clip(np.floor(c * 2097152.0), 0, 2097151).astype(np.uint32)
    key = tmx.hilbert_keys(q, 21)
    same = internal_region[1:] == internal_region[:-1]
    assert (key[1:][same] >= key[:-1][same]).all()
    starts = np.concatenate([[0], np.nonzero(~same)[0] + 1])
    assert (np.diff(key[starts].astype(np.float64)) > 0).all()


def test_face_entries(tmx):
    """Face entries: entry r of tet T is the face opposite T's vertex of rank r,
    holding the neighbour N across it and N's vertex opposite that face."""
    s = sg.make_config("tiny")
    m = tmx.Mesh(s.points, s.tets, s.tris, upload=False, faces=True)
    e = m.export()
    F = m.export_faces()
    V, Nb = e["cold"][:, :4], e["cold"][:, 4:]
    pts = e["points"].reshape(-1, 4)[:, :3]
    order = np.argsort(V, axis=1, kind="stable")
    for t in range(len(V)):
        for r in range(4):
            j = order[t, r]
            n = int(Nb[t, j])
            ent = F[t, r]
            assert ent[0] == n
            if n < 0:                       # flagged: constrained face or boundary
                assert ent[1] == -1
                continue
            face = set(V[t]) - {V[t, j]}
            w = (set(V[n]) - face).pop()
            assert len(set(V[n]) & face) == 3 and ent[1] == w
            assert np.array_equal(ent[2:5].view(np.float32), pts[w])
    with pytest.raises(Exception):
        tmx.Mesh(s.points, s.tets, s.tris, upload=False).export_faces()


def test_face16_entries(tmx):
    """16-byte face entries: the neighbour, the rank of its opposite vertex among
    its own ids (bits 29-30), and that vertex's position."""
    s = sg.make_config("tiny")
    m = tmx.Mesh(s.points, s.tets, s.tris, upload=False, faces=True, faces16=True)
    e = m.export()
    F = m.export_faces()
    G = m.export_faces16()
    V = e["cold"][:, :4]
    for t in range(len(V)):
        for r in range(4):
            n, w = int(F[t, r, 0]), int(F[t, r, 1])
            g = int(G[t, r, 0]) & 0xFFFFFFFF
            if n < 0:
                assert g == n & 0xFFFFFFFF
                continue
            assert g & 0x1FFFFFFF == n and g >> 31 == 0
            assert (g >> 29) & 3 == int((V[n] < w).sum())
            assert np.array_equal(G[t, r, 1:4], F[t, r, 2:5])


def test_restart_records(tmx):
    """Restart record of side s of triangle c: the tet the oracle's adjacency
    puts on that side, whose face opposite V[skip] is the triangle, with its
    cold record and its vertices' input positions inline."""
    s = sg.make_config("tiny")
    m = tmx.Mesh(s.points, s.tets, s.tris, upload=False)
    e = m.export()
    R = m.export_restart()
    _, _, ctet = oracle.OracleMesh(s.points, s.tets, s.tris).arrays()
    pperm, tperm = e["point_perm"], e["tet_perm"]
    assert R.shape == (len(s.tris), 2, 24)
    for c in range(len(s.tris)):
        tri = set(int(v) for v in s.tris[c])
        for side in range(2):
            r = R[c, side]
            T, skip = int(r[20]), int(r[21])
            if ctet[c, side] < 0:
                assert T == -1 and skip == -1
                continue
            assert tperm[T] == ctet[c, side]
            assert np.array_equal(r[0:8], e["cold"][T])
            V = r[0:4]
            assert set(int(pperm[V[k]]) for k in range(4) if k != skip) == tri
            xyz = r[8:20].view(np.float32).reshape(4, 3)
            assert np.array_equal(xyz, np.asarray(s.points, np.float32)[pperm[V]])
            assert r[22] == 0 and r[23] == 0


def test_restart_record_of_a_boundary_triangle(tmx):
    """A constrained triangle on the mesh boundary has a tet on one side only:
    that side's record names it, the other side's holds T = skip = -1."""
    pts, tets = sg.freudenthal_grid(3, 0.1, 7)
    nbr, _, _ = oracle.OracleMesh(pts, tets, np.zeros((0, 3), np.int32)).arrays()
    t, k = [int(x) for x in np.argwhere(nbr == -1)[0]]
    tri = np.array([[v for j, v in enumerate(tets[t]) if j != k]], np.int32)
    m = tmx.Mesh(pts, tets, tri, upload=False)
    e = m.export()
    R = m.export_restart()
    T = R[0, :, 20]
    assert sorted(T.tolist())[0] == -1 and (T >= 0).sum() == 1
    side = int(np.argmax(T >= 0))
    assert e["tet_perm"][T[side]] == t
    assert R[0, 1 - side, 21] == -1 and R[0, side, 21] >= 0
