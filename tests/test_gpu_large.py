"""Parity at the full size of the large workload: a 256^3-cell Kuhn grid
(100,663,296 tets, 1.1 M constrained triangles), 1024 x 1024 camera rays and
eight ambient-occlusion rays (t_max 0.05) per hit, traced in the launch
configuration the benchmark times (16-byte face entries, Hilbert order,
bounded walks for the occlusion rays).

The tet adjacency of this mesh is too large to build on the host in a test,
so the expected hits come from the oracle's brute force over all triangles
(the plain definition of the hit) on sampled rays; the side each ray arrives
from is taken from the geometry.  The device-generated occlusion rays of the
whole frame are checked by properties that hold at any size, and an even
sample of them by the brute force.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import scenegen as sg
from oracle.secondary import arrival_side, secondary_rays
from tests.parity import compare, hit_points

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AO_SEED = 0x5EED      # the benchmark's seed
AO_PER_HIT, AO_TMAX = 8, 0.05
N_PRIMARY, N_AO_PIXELS = 800, 300


@pytest.fixture(scope="module")
def tmx():
    from paper_2103_02309_gb300 import build
    build.build()
    from paper_2103_02309_gb300 import tetmesh
    return tetmesh


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def large(tmx):
    s = sg.make_config("large")
    mesh = tmx.Mesh(s.points, s.tets, s.tris, faces16=True)
    ts = oracle.OracleTriangles(s.points, s.tris)
    o, d = sg.camera_rays(s.camera)
    sel = np.random.default_rng(11).choice(len(d), N_PRIMARY, replace=False)
    w = ts.bruteforce(o[sel], d[sel], np.inf)
    # occlusion rays of the first sampled pixels, generated by the oracle from
    # its own hits (counter = pixel index, as on the device)
    k = slice(0, N_AO_PIXELS)
    side = arrival_side(s.points, s.tris, w["tri"][k], d[sel[k]])
    ob, db, tb, eb, _ = secondary_rays(s.points, s.tris, w["tri"][k], np.float32(w["b1"][k]),
                                       np.float32(w["b2"][k]), side, AO_SEED, AO_PER_HIT, AO_TMAX,
                                       ray_ids=sel[k])
    wb = ts.bruteforce(ob, db, tb, exclude=eb >> 1)
    return SimpleNamespace(s=s, mesh=mesh, ts=ts, sel=sel, w=w, ao=(ob, db, tb, eb), wb=wb)


@pytest.mark.parametrize("mode", ["fp32g", "fp64"])
def test_large_full_size_sampled(tmx, large, mode):
    L = large
    cam = L.s.camera
    assert L.mesh.info.n_tets == 100_663_296
    start = L.mesh.locate(torch.tensor([cam.eye], dtype=torch.float32, device="cuda"))
    rays = tmx.gen_primary(tmx.make_camera(cam.eye, cam.fov_deg, cam.width, cam.height), start)
    op = tmx.trace_opts(mode=mode)
    ob = tmx.trace_opts(mode=mode, tmax_early_exit=True)
    hits = L.mesh.trace(rays, opts=op)
    r2, cnt, _ = L.mesh.gen_secondary(hits, AO_PER_HIT, AO_TMAX, seed=AO_SEED)
    h2 = L.mesh.trace(r2, n_dev=cnt, opts=ob)
    torch.cuda.synchronize()

    g = tmx.unpack_hits(hits[torch.from_numpy(L.sel).cuda()])
    st = compare(L.s.points, L.s.tris, g, L.w)
    assert (L.w["tri"] >= 0).mean() > 0.9

    o3, d3, t3, e3 = L.ao
    gb = tmx.unpack_hits(L.mesh.trace(dev(tmx.pack_rays(o3, d3, t3, -1 - e3)), opts=ob))
    st2 = compare(L.s.points, L.s.tris, gb, L.wb)
    assert st2["hits"] > 0.05 * len(o3)
    assert (gb["t"][gb["tri"] >= 0] <= AO_TMAX).all()

    # the occlusion rays of the whole frame, as generated on the device
    k = int(cnt.item())
    n_hit = int((tmx.unpack_hits(hits)["tri"] >= 0).sum())
    assert k == AO_PER_HIT * n_hit
    sel2 = np.random.default_rng(12).choice(k, min(k, 200000), replace=False)
    idx = torch.from_numpy(sel2).cuda()
    rb = r2[idx].cpu().numpy()
    g2 = tmx.unpack_hits(h2[idx])
    hit = g2["tri"] >= 0
    assert 0.05 < hit.mean() < 0.95
    assert (g2["t"][hit] > 0).all() and (g2["t"][hit] <= AO_TMAX).all()
    on_ray = rb[hit, 0:3].astype(np.float64) + g2["t"][hit, None].astype(np.float64) * rb[hit, 4:7]
    on_tri = hit_points(L.s.points, L.s.tris, g2["tri"][hit], g2["b1"][hit], g2["b2"][hit])
    assert np.linalg.norm(on_ray - on_tri, axis=1).max() < 4e-6
    assert (g2["b1"][hit] >= -1e-5).all() and (g2["b2"][hit] >= -1e-5).all()
    assert (g2["b1"][hit] + g2["b2"][hit] <= 1 + 1e-5).all()
    # and an even sample of them against the oracle's brute force, each from
    # its restart face
    pick = np.sort(sel2)[:: max(1, len(sel2) // 3000)]
    rp = r2[torch.from_numpy(pick).cuda()].cpu().numpy()
    gp = tmx.unpack_hits(h2[torch.from_numpy(pick).cuda()])
    ep = -1 - rp.view(np.int32)[:, 3]
    wp = L.ts.bruteforce(rp[:, 0:3], rp[:, 4:7], rp[:, 7], exclude=ep >> 1)
    st3 = compare(L.s.points, L.s.tris, gp, wp)
    print(mode, "primary", st, "ao", st2, "device ao", st3)


def test_large_scene_at_128_cells_every_ray(tmx):
    """The large workload's scene reduced to 128^3 cells (12.6 M tets, a size
    whose adjacency the oracle builds): every camera ray of the 1024 x 1024
    frame and every one of the 8.39 M occlusion rays the device generates
    from its hits, walked as the benchmark walks them (bounded walks that
    stop at t_max), against the oracle's walk from each ray's start tet or
    restart face."""
    from tests.test_gpu_parity import camera_case
    c = camera_case(tmx, "large", n_override=128)
    cam = c.s.camera
    assert cam.width * cam.height == 1024 * 1024
    start = dev(np.array([c.cam_internal], np.int32))
    rays = tmx.gen_primary(tmx.make_camera(cam.eye, cam.fov_deg, cam.width, cam.height), start)
    hits = c.mesh.trace(rays)
    r2, cnt, _ = c.mesh.gen_secondary(hits, AO_PER_HIT, AO_TMAX, seed=AO_SEED)
    h2 = c.mesh.trace(r2, n_dev=cnt, tmax_early_exit=True)
    torch.cuda.synchronize()
    o, d = sg.camera_rays(cam)
    g = tmx.unpack_hits(hits)
    st = compare(c.s.points, c.s.tris, g, c.oracle_trace(o, d, np.inf, c.cam_in[0]))
    k = int(cnt.item())
    assert k == AO_PER_HIT * int((g["tri"] >= 0).sum())
    rb = r2[:k].cpu().numpy()
    g2 = tmx.unpack_hits(h2[:k])
    entry = -1 - rb.view(np.int32)[:, 3]
    st2 = compare(c.s.points, c.s.tris, g2, c.oracle_trace(rb[:, 0:3], rb[:, 4:7], rb[:, 7], -1, entry))
    assert st2["hits"] > 1000 and st2["n"] - st2["hits"] > 1000     # occluded and open rays
    print("primary", st, "occlusion", st2)
