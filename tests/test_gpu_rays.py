"""Shadow, reflection and refraction rays (Sec. 6) on the CUDA path against the oracle.

The rays each side traces come from the oracle's generators applied to the
oracle's own primary hits; the device generators get those same hits as
input and are compared with the oracle's generators ray by ray.
"""
import numpy as np
import pytest

import scenegen as sg
from oracle.secondary import hit_side, shadow_rays, specular_rays
from tests.parity import compare
from tests.test_gpu_parity import camera_case, dev, device_hits, tmx  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# point lights placed so that both lit and shadowed hit points occur
LIGHTS = {"tiny": (0.05, 0.5, 0.23), "medium": (0.1, 0.55, 0.28)}
LIGHT = LIGHTS["tiny"]


def oracle_primary(c):
    """Oracle hits of the camera rays of case c, and the rays."""
    o, d = sg.camera_rays(c.s.camera)
    w = c.oracle_trace(o, d, np.inf, c.cam_in[0])
    return o, d, w


def light_tet(c, L):
    t, margin = c.om.locate(np.array([L], np.float32))
    assert margin[0] > 1e-4, "light too close to a face of its tet"
    return int(t[0]), int(c.tinv[t[0]])


@pytest.fixture(scope="module")
def tiny(tmx):
    return camera_case(tmx, "tiny")


@pytest.fixture(scope="module")
def medium(tmx):
    """The 16-sphere scene on a 24^3 grid, seen by a 320x180 camera."""
    import dataclasses

    from tests.test_gpu_parity import Case
    s = sg.make_config("medium", n_override=24)
    s = dataclasses.replace(s, camera=sg.Camera(s.camera.eye, s.camera.fov_deg, 320, 180))
    c = Case(tmx, s)
    c.cam_in, mb = c.om.locate(np.array([s.camera.eye], np.float32))
    assert mb[0] > 1e-9
    c.cam_internal = int(c.tinv[c.cam_in[0]])
    return c


def test_gen_shadow_matches_oracle(tmx, tiny):
    c = tiny
    o, d, w = oracle_primary(c)
    h, _ = device_hits(tmx, c, w)
    B = np.float32(w["b1"]), np.float32(w["b2"])
    r, cnt, src = c.mesh.gen_shadow(dev(h), LIGHT, src=True)
    torch.cuda.synchronize()
    k = int(cnt.item())
    r = r[:k].cpu().numpy()
    src = src[:k].cpu().numpy()
    o2, d2, tm2, entry, src_o = shadow_rays(c.s.points, c.s.tris, w["tri"], *B, LIGHT)
    assert k == len(o2) == (w["tri"] >= 0).sum() > 100
    assert np.array_equal(src, src_o)
    assert np.abs(r[:, 0:3] - o2).max() < 1e-6
    assert np.abs(r[:, 4:7] - d2).max() < 2e-6
    assert np.abs(r[:, 7] / tm2 - 1).max() < 2e-6
    # the facing side agrees wherever the light is not within rounding of the plane
    P = c.s.points.astype(np.float64)
    t = c.s.tris[w["tri"][src_o]]
    nrm = np.cross(P[t[:, 1]] - P[t[:, 0]], P[t[:, 2]] - P[t[:, 0]])
    lv = np.asarray(LIGHT) - P[t[:, 0]]
    clear = np.abs(np.einsum("ij,ij->i", nrm, lv)) > 1e-5 * np.linalg.norm(nrm, axis=1) * np.linalg.norm(lv, axis=1)
    assert clear.mean() > 0.99
    assert np.array_equal((-1 - r.view(np.int32)[:, 3])[clear], entry[clear])


@pytest.mark.parametrize("mode", ["fp32g", "fp32", "fp64"])
@pytest.mark.parametrize("scene", ["tiny", "medium"])
def test_shadow_trace_matches_oracle(tmx, request, scene, mode):
    c = request.getfixturevalue(scene)
    o, d, w = oracle_primary(c)
    L = LIGHTS[scene]
    o2, d2, tm2, entry, _ = shadow_rays(c.s.points, c.s.tris, w["tri"], np.float32(w["b1"]),
                                        np.float32(w["b2"]), L)
    _, lt = light_tet(c, L)
    rays = dev(tmx.pack_rays(o2, d2, tm2, -1 - entry))
    g = tmx.unpack_hits(c.mesh.trace_shadow(rays, dev(np.array([lt], np.int32)), mode=mode))
    wo = c.oracle_trace(o2, d2, tm2, -1, entry)
    st = compare(c.s.points, c.s.tris, g, wo, check_t=(mode != "fp32"))
    reached = (g["flags"] & tmx.HIT_REACHED) != 0
    assert not reached[g["tri"] >= 0].any()
    lit = (wo["tri"] < 0) & (g["tri"] < 0)
    assert lit.sum() > 50 and (wo["tri"] >= 0).sum() > 50   # both lit and shadowed points
    assert reached[lit].mean() > 0.999
    assert (g["tet"][reached] == lt).all()
    print(scene, mode, st, "lit", int(lit.sum()))


def test_shadow_ray_from_inside_the_light_tet(tmx, tiny):
    c = tiny
    t_in, lt = light_tet(c, LIGHT)
    q = np.array([LIGHT], np.float32) + np.float32(1e-4)
    tq, mq = c.om.locate(q)
    assert tq[0] == t_in and mq[0] > 1e-6
    d = np.array([[0.3, -0.2, 0.9]], np.float32)
    d /= np.linalg.norm(d)
    rays = dev(tmx.pack_rays(q, d, 1e-3, np.array([lt], np.int32)))
    g = tmx.unpack_hits(c.mesh.trace_shadow(rays, dev(np.array([lt], np.int32))))
    assert g["tri"][0] == -1 and g["flags"][0] & tmx.HIT_REACHED and g["steps"][0] == 0


@pytest.mark.parametrize("kind,ior", [("reflect", 1.5), ("refract", 1.5), ("refract", 1 / 1.5)])
def test_gen_specular_matches_oracle(tmx, tiny, kind, ior):
    c = tiny
    o, d, w = oracle_primary(c)
    h, side = device_hits(tmx, c, w)
    rin = dev(tmx.pack_rays(o, d, np.inf, c.cam_internal))
    r, cnt, src = c.mesh.gen_specular(rin, dev(h), kind, ior, tmax=7.0, src=True)
    torch.cuda.synchronize()
    k = int(cnt.item())
    r = r[:k].cpu().numpy()
    src = src[:k].cpu().numpy()
    o2, d2, tm2, entry, src_o, kk = specular_rays(c.s.points, c.s.tris, w["tri"], np.float32(w["b1"]),
                                                  np.float32(w["b2"]), side, d, kind, ior, 7.0)
    assert k == len(o2) > 100
    assert np.array_equal(src, src_o)
    assert np.abs(r[:, 0:3] - o2).max() < 1e-6
    assert np.array_equal(r[:, 7], tm2)
    clear = np.abs(kk) > 1e-3          # away from the onset of total internal reflection
    assert clear.mean() > 0.95
    assert np.array_equal((-1 - r.view(np.int32)[:, 3])[clear], entry[clear])
    assert np.abs(r[clear, 4:7] - d2[clear]).max() < 2e-5


@pytest.mark.parametrize("kind,ior", [("reflect", 1.5), ("refract", 1.5), ("refract", 1 / 1.5)])
def test_specular_trace_matches_oracle(tmx, medium, kind, ior):
    c = medium
    o, d, w = oracle_primary(c)
    side = hit_side(c.ctet, w["tri"], w["tet"])
    o2, d2, tm2, entry, _, _ = specular_rays(c.s.points, c.s.tris, w["tri"], np.float32(w["b1"]),
                                             np.float32(w["b2"]), side, d, kind, ior, np.inf)
    rays = dev(tmx.pack_rays(o2, d2, tm2, -1 - entry))
    for mode in ("fp32g", "fp64"):
        g = tmx.unpack_hits(c.mesh.trace(rays, mode=mode))
        wo = c.oracle_trace(o2, d2, tm2, -1, entry)
        st = compare(c.s.points, c.s.tris, g, wo)
        assert st["hits"] > 100
        print(kind, ior, mode, st)
