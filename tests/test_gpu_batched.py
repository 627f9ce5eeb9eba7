"""Parity at the full size of the batched workload: 32 uneven meshes
(16^3..96^3 cells, 27.8 M tets), about 6.9 M rays, half of each mesh's rays
from a camera and half in uniform directions from interior points, traced in
one persistent graph-replayed launch with the settings the autotuner picks,
as the benchmark times it.

Rays are made on the host by the scene generator (the device's primary-ray
generator is bit-exact with it, see test_gen_primary_bit_exact); only their
start tets come from the device's point location, which the oracle does not
use.  Expected hits: the oracle's brute force over all triangles of each
mesh, on sampled rays.  Every ray: the batch equals one launch per mesh.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests.parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SAMPLES_PER_MESH = 2000


@pytest.fixture(scope="module")
def tmx():
    from paper_2103_02309_gb300 import build
    build.build()
    from paper_2103_02309_gb300 import tetmesh
    return tetmesh


def test_batched_full_size_sampled(tmx):
    descs = sg.batched_meshes()
    assert len(descs) == 32
    meshes, rays, hits, host = [], [], [], []
    for dsc in descs:
        s = sg.make_grid_scene("batched", dsc["n"], sg.BATCHED["jitter"], dsc["seed"],
                               n_spheres=dsc["n_spheres"])
        mesh = tmx.Mesh(s.points, s.tets, s.tris, faces=True, faces16=True)
        n_prim = dsc["primary"]
        side = max(1, int(math.ceil(math.sqrt(n_prim))))
        cam = sg.Camera(sg.BATCHED["camera_eye"], sg.BATCHED["fov_deg"], side,
                        max(1, int(math.ceil(n_prim / side))))
        o1, d1 = sg.camera_rays(cam)
        n_uni = dsc["rays"] - n_prim
        o2 = sg.interior_points(n_uni, dsc["seed"])
        d2 = sg.uniform_directions(n_uni, dsc["seed"])
        o = np.concatenate([o1, o2]).astype(np.float32)
        d = np.concatenate([d1, d2]).astype(np.float32)
        eye = mesh.locate(torch.tensor([sg.BATCHED["camera_eye"]], dtype=torch.float32,
                                       device="cuda"))
        start = torch.cat([eye.expand(len(o1)),
                           mesh.locate(torch.from_numpy(o2).cuda())]).cpu().numpy()
        assert (start >= 0).all()
        r = torch.from_numpy(tmx.pack_rays(o, d, np.inf, start)).cuda()
        meshes.append(mesh)
        rays.append(r)
        hits.append(torch.empty((len(o), 8), dtype=torch.int32, device="cuda"))
        host.append((s.points, s.tris, o, d))
    assert 27_000_000 < sum(m.info.n_tets for m in meshes) < 29_000_000
    assert sum(len(h[2]) for h in host) > 5_000_000

    b = tmx.Batch(meshes)
    b.set(rays, hits)
    tuned = b.autotune(reps=1)
    b.run()
    torch.cuda.synchronize()
    got = [tmx.unpack_hits(h) for h in hits]

    # every ray: the batch equals one launch per mesh
    for h in hits:
        h.fill_(-7)
    b.run_separate()
    torch.cuda.synchronize()
    for g, h in zip(got, hits):
        sep = tmx.unpack_hits(h)
        for k in ("tri", "t", "b1", "b2", "tet", "steps"):
            assert np.array_equal(g[k], sep[k]), k

    # sampled rays of every mesh against the brute-force oracle
    g_rng = np.random.default_rng(17)
    stats = []
    for (pts, tris, o, d), g in zip(host, got):
        idx = g_rng.choice(len(o), min(SAMPLES_PER_MESH, len(o)), replace=False)
        w = oracle.OracleTriangles(pts, tris).bruteforce(o[idx], d[idx], np.inf)
        stats.append(compare(pts, tris, {k: v[idx] for k, v in g.items()}, w))
    b.close()
    print("autotuned", tuned.opts.format, tuned.opts.block, tuned.opts.refill,
          tuned.opts.batch_steps, tuned.sort_chunk,
          "rays compared", sum(st["n"] for st in stats),
          "hits", sum(st["hits"] for st in stats),
          "mismatches", sum(st["mismatches"] for st in stats))
