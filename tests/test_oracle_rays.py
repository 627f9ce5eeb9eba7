"""Pins of the oracle's shadow, reflection and refraction ray generators
(Sec. 6) against geometry and Snell's law, checked with formulas of their own.
"""
import numpy as np
import pytest

import oracle.secondary as gen


def scene(seed, m=4000):
    """Random triangles, hits inside them (some misses), incoming directions."""
    g = np.random.default_rng(seed)
    pts = g.uniform(0, 1, size=(3 * m, 3)).astype(np.float32)
    tris = np.arange(3 * m, dtype=np.int32).reshape(m, 3)
    hit_tri = np.where(g.random(m) < 0.8, np.arange(m), -1).astype(np.int32)
    u = g.uniform(0.05, 0.9, size=(m, 2))
    u = np.where(u.sum(1, keepdims=True) < 0.95, u, u * 0.45)
    side = (g.random(m) < 0.5).astype(np.int32)
    P = pts.astype(np.float64)
    n = np.cross(P[tris[:, 1]] - P[tris[:, 0]], P[tris[:, 2]] - P[tris[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    na = np.where(side[:, None] == 1, -n, n)
    # incoming directions travel against the arrival side's normal
    w = g.normal(size=(m, 3))
    flip = np.einsum("ij,ij->i", w, na) > 0
    w[flip] *= -1
    return pts, tris, hit_tri, u[:, 0].astype(np.float32), u[:, 1].astype(np.float32), side, w, n


def check_shadow(m):
    pts, tris, hit_tri, b1, b2, _, _, _ = scene(1)
    L = np.array([0.3, 1.4, -0.2])
    o, d, tmax, entry, src = m.shadow_rays(pts, tris, hit_tri, b1, b2, L)
    assert np.array_equal(src, np.nonzero(hit_tri >= 0)[0])
    end = o.astype(np.float64) + tmax[:, None].astype(np.float64) * d.astype(np.float64)
    assert np.abs(end - L).max() < 4e-6
    assert np.abs(np.linalg.norm(d.astype(np.float64), axis=1) - 1).max() < 1e-6
    P = pts.astype(np.float64)
    c = hit_tri[src]
    M = np.stack([P[tris[c, 1]] - P[tris[c, 0]], P[tris[c, 2]] - P[tris[c, 0]],
                  np.broadcast_to(L, (len(c), 3)) - P[tris[c, 0]]], axis=1)
    faces = np.linalg.det(M) >= 0          # the light is on the + side
    assert np.array_equal(entry, 2 * c + np.where(faces, 0, 1))
    # the ray starts into the side of the light: d points to that side
    n = np.cross(M[:, 0], M[:, 1])
    dn = np.einsum("ij,ij->i", d.astype(np.float64), n)
    assert ((dn > 0) == faces)[np.abs(dn) > 1e-6].all()


def check_reflect(m):
    pts, tris, hit_tri, b1, b2, side, w, n = scene(2)
    o, d, _, entry, src, _ = m.specular_rays(pts, tris, hit_tri, b1, b2, side, w, "reflect", 1.5, 1.0)
    w = w[src] / np.linalg.norm(w[src], axis=1, keepdims=True)
    n = n[src]
    d = d.astype(np.float64)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-6
    # equal angles: the normal component flips, the tangential one stays
    assert np.abs(np.einsum("ij,ij->i", d, n) + np.einsum("ij,ij->i", w, n)).max() < 1e-6
    tw = w - np.einsum("ij,ij->i", w, n)[:, None] * n
    td = d - np.einsum("ij,ij->i", d, n)[:, None] * n
    assert np.abs(tw - td).max() < 1e-6
    assert np.array_equal(entry, 2 * hit_tri[src] + side[src])


def check_refract(m, ior):
    pts, tris, hit_tri, b1, b2, side, w, n = scene(3)
    o, d, _, entry, src, k = m.specular_rays(pts, tris, hit_tri, b1, b2, side, w, "refract", ior, 1.0)
    w = w[src] / np.linalg.norm(w[src], axis=1, keepdims=True)
    n = n[src]
    s = side[src]
    d = d.astype(np.float64)
    eta = np.where(s == 1, ior, 1 / ior)    # arrival-side index over far-side index
    sin_i = np.linalg.norm(np.cross(w, n), axis=1)
    sin_t = np.linalg.norm(np.cross(d, n), axis=1)
    tir = eta * sin_i > 1
    clear = np.abs(eta * sin_i - 1) > 1e-6
    assert tir.any() == (ior != 1) and (~tir).any()
    assert np.array_equal((k < 0)[clear], tir[clear])
    ok = ~tir & clear
    assert np.abs(sin_t[ok] - eta[ok] * sin_i[ok]).max() < 2e-6          # Snell
    assert np.abs(np.einsum("ij,ij->i", np.cross(w, n), d)).max() < 2e-6  # plane of incidence
    # transmitted rays cross to the far side; reflected ones stay
    nd, nw = np.einsum("ij,ij->i", d, n), np.einsum("ij,ij->i", w, n)
    assert (np.sign(nd[ok]) == np.sign(nw[ok])).all()
    tt = tir & clear
    assert (np.sign(nd[tt]) == -np.sign(nw[tt])).all()
    c = hit_tri[src]
    assert np.array_equal(entry[ok], (2 * c + 1 - s)[ok])
    assert np.array_equal(entry[tt], (2 * c + s)[tt])


def check_special(m):
    pts, tris, hit_tri, b1, b2, side, w, n = scene(4, 500)
    # equal indices: the ray goes straight through
    _, d, _, entry, src, _ = m.specular_rays(pts, tris, hit_tri, b1, b2, side, w, "refract", 1.0, 1.0)
    ww = w[src] / np.linalg.norm(w[src], axis=1, keepdims=True)
    assert np.abs(d - ww).max() < 1e-6
    assert np.array_equal(entry, 2 * hit_tri[src] + 1 - side[src])
    # normal incidence: no bending for any index ratio
    na = np.where(side[:, None] == 1, -n, n)
    _, d, _, _, src, _ = m.specular_rays(pts, tris, hit_tri, b1, b2, side, -na, "refract", 1.7, 1.0)
    assert np.abs(d + na[src]).max() < 1e-6


CHECKS = [check_shadow, check_reflect, lambda m: check_refract(m, 1.5),
          lambda m: check_refract(m, 1 / 1.33), check_special]


def test_shadow_rays_reach_the_light():
    check_shadow(gen)


def test_reflection_mirrors_about_the_normal():
    check_reflect(gen)


@pytest.mark.parametrize("ior", [1.5, 1 / 1.33])
def test_refraction_follows_snell(ior):
    check_refract(gen, ior)


def test_refraction_special_cases():
    check_special(gen)
