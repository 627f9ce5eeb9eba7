"""Pins of two readings of the paper, in plain numpy (no product or oracle code).

R1 (Alg. 1, Sec. 4): with det(a, b) = a.x*b.y - a.y*b.x and the entry face
p0, p1, p2 counter-clockwise around the origin, GetExitFace returns the slot
that the new vertex replaces, and the face kept is counter-clockwise again.
R3 (Eq. 1-2): the scaled basis with v = t / |t_min| is orthogonal to d, has
u_min = 0, u_other = +-1, v_min = +-1, and (u, v, d) is right-handed, so
every 2-D sign test agrees with the one in an orthonormal right-handed basis.
"""
import numpy as np


def alg1(p0, p1, p2, p3):
    def det(a, b):
        return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]
    e = np.zeros(len(p0), np.int64)
    neg0 = det(p3, p0) < 0
    e = np.where(neg0 & (det(p3, p2) >= 0), 1, e)
    e = np.where(~neg0 & (det(p3, p1) < 0), 2, e)
    return e


def scaled_basis(d):
    """Eq. 1-2 with v = t / |t_min| (reading R3), per row of d (float64)."""
    a = np.abs(d)
    n = len(d)
    mn = np.argmin(a, axis=1)                                  # lowest index of the smallest
    mx = 2 - np.argmax(a[:, ::-1], axis=1)                     # highest index of the largest
    rows = np.arange(n)
    i1, i2 = (mn + 1) % 3, (mn + 2) % 3
    dmx = d[rows, mx]
    u = np.zeros_like(d)
    u[rows, i1] = d[rows, i2] / dmx
    u[rows, i2] = -d[rows, i1] / dmx
    t = np.cross(d, u)
    v = t / np.abs(t[rows, mn])[:, None]
    return u, v, mn, mx


def random_entry_configs(count, seed):
    g = np.random.default_rng(seed)
    a, b, c = (g.normal(size=(count, 3)) for _ in range(3))
    n = np.cross(b - a, c - a)
    nh = n / np.linalg.norm(n, axis=1, keepdims=True)
    w = g.dirichlet([1, 1, 1], size=count)
    O = w[:, :1] * a + w[:, 1:2] * b + w[:, 2:] * c           # origin inside the entry face
    lat = 0.7 * g.normal(size=(count, 3))
    lat -= (lat * nh).sum(1, keepdims=True) * nh               # keep x on the + side of the face
    x = (a + b + c) / 3 + lat + nh * g.uniform(0.2, 2.0, (count, 1))
    d = g.normal(size=(count, 3))
    d = np.where(((d * nh).sum(1) < 0)[:, None], -d, d)        # into the tet through (a, b, c)
    return a, b, c, x, O, d


def exit_face_3d(a, b, c, x, O, d):
    """Which of the faces (x,b,c), (a,x,c), (a,b,x) the ray leaves through (0, 1, 2), by
    intersecting it with the three triangles."""
    out = np.full(len(a), -1)
    faces = [(x, b, c), (a, x, c), (a, b, x)]
    for k, (p, q, r) in enumerate(faces):
        e1, e2 = q - p, r - p
        pv = np.cross(d, e2)
        det = (e1 * pv).sum(1)
        s = O - p
        u = (s * pv).sum(1) / det
        qv = np.cross(s, e1)
        v = (d * qv).sum(1) / det
        t = (e2 * qv).sum(1) / det
        inside = (u > 1e-9) & (v > 1e-9) & (u + v < 1 - 1e-9) & (t > 1e-12)
        out = np.where(inside, k, out)
    return out


def test_alg1_exit_slot_with_counter_clockwise_entry_face():
    a, b, c, x, O, d = random_entry_configs(200_000, 1)
    want = exit_face_3d(a, b, c, x, O, d)
    ok = want >= 0                                            # drop near-degenerate draws
    assert ok.mean() > 0.99
    u, v, _, _ = scaled_basis(d)

    def proj(p):
        q = p - O
        return np.stack([(u * q).sum(1), (v * q).sum(1)], 1)
    P = [proj(a), proj(b), proj(c)]
    p3 = proj(x)
    det01 = P[0][:, 0] * P[1][:, 1] - P[0][:, 1] * P[1][:, 0]
    ccw = det01 > 0
    # order the entry face counter-clockwise: swap slots 1 and 2 where needed
    slot_label = np.where(ccw[:, None], [0, 1, 2], [0, 2, 1])
    q0 = P[0]
    q1 = np.where(ccw[:, None], P[1], P[2])
    q2 = np.where(ccw[:, None], P[2], P[1])
    e = alg1(q0, q1, q2, p3)
    replaced = slot_label[np.arange(len(e)), e]               # entry-face vertex replaced by x
    assert (replaced[ok] == want[ok]).all()
    # the kept face (p3 in slot e) is counter-clockwise again
    Q = np.stack([q0, q1, q2], 1)
    Q[np.arange(len(e)), e] = p3
    d01 = Q[:, 0, 0] * Q[:, 1, 1] - Q[:, 0, 1] * Q[:, 1, 0]
    d12 = Q[:, 1, 0] * Q[:, 2, 1] - Q[:, 1, 1] * Q[:, 2, 0]
    d20 = Q[:, 2, 0] * Q[:, 0, 1] - Q[:, 2, 1] * Q[:, 0, 0]
    assert ((d01 > 0) & (d12 > 0) & (d20 > 0))[ok].mean() > 0.9999
    # with the opposite (clockwise) order Alg. 1 is wrong for most rays
    e_cw = alg1(q0, q2, q1, p3)
    lab_cw = np.where(ccw[:, None], [0, 2, 1], [0, 1, 2])[np.arange(len(e)), e_cw]
    assert (lab_cw[ok] == want[ok]).mean() < 0.7


def test_scaled_basis_identities():
    g = np.random.default_rng(2)
    d = g.normal(size=(100_000, 3))
    special = np.array([[1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 1], [1, -1, 0], [0, 2, 2],
                        [3, 3, -1], [-1e-30, 1, 0.5]], float)
    d = np.concatenate([d, special])
    u, v, mn, mx = scaled_basis(d)
    rows = np.arange(len(d))
    other = 3 - mn - mx
    assert (u[rows, mn] == 0).all()
    assert (np.abs(u[rows, other]) == 1).all()
    assert (np.abs(v[rows, mn]) == 1).all()
    assert (np.abs(u) <= 1).all() and (np.abs(v) <= 1 + 1e-15).all()
    nd = np.linalg.norm(d, axis=1)
    assert (np.abs((u * d).sum(1)) <= 1e-15 * nd * np.linalg.norm(u, axis=1)).all()
    assert (np.abs((v * d).sum(1)) <= 1e-15 * nd * np.linalg.norm(v, axis=1)).all()
    assert (np.einsum("ij,ij->i", np.cross(u, v), d) > 0).all()       # right-handed
    # every 2-D sign test agrees with an orthonormal right-handed basis (Duff et al. 2017)
    dh = d / nd[:, None]
    s = np.where(dh[:, 2] >= 0, 1.0, -1.0)
    aa = -1.0 / (s + dh[:, 2])
    bb = dh[:, 0] * dh[:, 1] * aa
    e1 = np.stack([1 + s * dh[:, 0] ** 2 * aa, s * bb, -s * dh[:, 0]], 1)
    e2 = np.stack([bb, s + dh[:, 1] ** 2 * aa, -dh[:, 1]], 1)
    hand = np.sign(np.einsum("ij,ij->i", np.cross(e1, e2), dh))
    p, q = g.normal(size=(len(d), 3)), g.normal(size=(len(d), 3))

    def det2(b1, b2):
        return (b1 * p).sum(1) * (b2 * q).sum(1) - (b2 * p).sum(1) * (b1 * q).sum(1)
    ours, ref = det2(u, v), det2(e1, e2) * hand
    big = np.abs(ref) > 1e-9
    assert (np.sign(ours[big]) == np.sign(ref[big])).all()
