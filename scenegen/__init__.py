"""Seeded synthetic scenes for constrained tet-mesh ray traversal.

This module only *generates inputs*: points, tetrahedra, constrained
triangles, cameras and rays.  It holds none of the traversal arithmetic
(no exit-face tests, no adjacency, no Hilbert order, no hit computation),
so that both the FP64 oracle and the CUDA path can be fed from it without
sharing any of the method's code.

Scene recipe (stands in for the paper's TetGen meshes of Sec. 8, which are
not available):

* Freudenthal / Kuhn grid over [0,1]^3 with n cubes per axis, h = 1/n.
  Point (i,j,k) has id i + (n+1)*(j + (n+1)*k) ("lexicographic, i fastest").
  Interior points get an independent uniform offset in [-jitter*h, +jitter*h]
  per axis; points on the hull stay exactly on the grid, so the hull is the
  unit cube.  Each cube (i,j,k) (id c = i + n*(j + n*k)) is split into the
  6 tetrahedra v000 -> +e_a -> +e_a+e_b -> v111 for the axis permutations
  (a,b,c) in lexicographic order; tet id = 6*c + permutation index.  Odd
  permutations swap their last two vertices so that every tet is positively
  oriented: orient3d(V0,V1,V2,V3) = det[V1-V0, V2-V0, V3-V0] > 0.
* A cell is "inside" when its undisplaced centre lies strictly inside the
  union of spheres.  Every cell face between an inside and an outside cell
  becomes two constrained triangles, split along the face diagonal from its
  minimum to its maximum corner (the diagonal the Kuhn split puts there):
  (q00, q10, q11) and (q00, q11, q01), with b < c the two in-face axes,
  each with its last two vertices swapped where needed so that its normal
  (v1-v0) x (v2-v0) points out of the inside cell (the "+ side" is outside).
  Triangle id = enumeration order: axis (x, y, z), then face position with
  i fastest, then the half.
* Pinhole camera looking along +z, image x along +x, image y (downwards)
  along -y, field of view across the shorter image side, pixel centres at
  (px+0.5, py+0.5).  Directions are formed and normalised with a fixed chain
  of correctly rounded float32 operations (see camera_rays).  Rays are stored in warp tiles of 8x4 pixels,
  tiles in row-major order, pixels row-major inside a tile (ragged edge
  tiles keep only in-image pixels).

Every random draw uses numpy's Philox counter-based generator with the
seed recorded in the config.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

TILE_W = 8
TILE_H = 4

# Axis permutations in lexicographic order; the tet id inside a cube is the
# index into this list.
_PERMS = list(permutations(range(3)))
_PERM_ODD = [((p[0] > p[1]) + (p[0] > p[2]) + (p[1] > p[2])) % 2 == 1 for p in _PERMS]


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def point_id(n: int, i, j, k):
    m = n + 1
    return i + m * (j + m * k)


def freudenthal_grid(n: int, jitter: float, seed: int):
    """Points (float32 [(n+1)^3, 3]) and positively oriented tets (int32 [6n^3, 4])."""
    m = n + 1
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    pts = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64) * h
    if jitter > 0.0:
        interior = ((i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < n)).ravel()
        off = _rng(seed, 0).uniform(-jitter * h, jitter * h, size=(m ** 3, 3))
        pts[interior] += off[interior]
    pts32 = pts.astype(np.float32)

    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v000 = point_id(n, ci.ravel(), cj.ravel(), ck.ravel()).astype(np.int64)
    step = np.array([1, m, m * m], dtype=np.int64)
    v111 = v000 + step.sum()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for pi, (a, b, _c) in enumerate(_PERMS):
        v1 = v000 + step[a]
        v2 = v1 + step[b]
        if _PERM_ODD[pi]:
            tets[:, pi] = np.stack([v000, v1, v111, v2], axis=1)
        else:
            tets[:, pi] = np.stack([v000, v1, v2, v111], axis=1)
    return pts32, tets.reshape(-1, 4).astype(np.int32)


def random_spheres(count: int, seed: int):
    """Centres uniform in [0.15, 0.85]^3, radii uniform in [0.03, 0.12]."""
    g = _rng(seed, 1)
    centres = g.uniform(0.15, 0.85, size=(count, 3))
    radii = g.uniform(0.03, 0.12, size=count)
    return centres, radii


def inside_cells(n: int, centres, radii) -> np.ndarray:
    """bool [n, n, n] indexed [k, j, i]: undisplaced cell centre strictly inside a sphere."""
    h = 1.0 / n
    inside = np.zeros((n, n, n), dtype=bool)
    for c, r in zip(np.asarray(centres, dtype=np.float64), np.asarray(radii, dtype=np.float64)):
        lo = np.maximum(np.floor((c - r) / h - 0.5).astype(int) - 1, 0)
        hi = np.minimum(np.ceil((c + r) / h - 0.5).astype(int) + 2, n)
        xs = (np.arange(lo[0], hi[0]) + 0.5) * h
        ys = (np.arange(lo[1], hi[1]) + 0.5) * h
        zs = (np.arange(lo[2], hi[2]) + 0.5) * h
        d2 = ((zs[:, None, None] - c[2]) ** 2 + (ys[None, :, None] - c[1]) ** 2
              + (xs[None, None, :] - c[0]) ** 2)
        inside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= d2 < r * r
    return inside


def slab_cells(n: int, layer: int) -> np.ndarray:
    """Cells with k < layer are 'inside': one constrained plane z = layer*h."""
    inside = np.zeros((n, n, n), dtype=bool)
    inside[:layer] = True
    return inside


def constrained_faces(n: int, inside: np.ndarray) -> np.ndarray:
    """Triangles (int32 [Nc, 3], grid point ids) between inside and outside cells."""
    out = []
    for axis in range(3):  # 0 = x (array axis 2), 1 = y (axis 1), 2 = z (axis 0)
        arr_axis = 2 - axis
        a = np.take(inside, np.arange(n - 1), axis=arr_axis)
        b = np.take(inside, np.arange(1, n), axis=arr_axis)
        kk, jj, ii = np.nonzero(a != b)
        base = [ii.astype(np.int64), jj.astype(np.int64), kk.astype(np.int64)]
        base[axis] = base[axis] + 1  # the face lies on the far side of the lower cell
        bax, cax = [ax for ax in range(3) if ax != axis]
        def pid(db, dc):
            q = list(base)
            q[bax] = q[bax] + db
            q[cax] = q[cax] + dc
            return point_id(n, q[0], q[1], q[2])
        q00, q10, q01, q11 = pid(0, 0), pid(1, 0), pid(0, 1), pid(1, 1)
        # (q10 - q00) x (q11 - q00) points along +axis for x and z, -axis for
        # y; flip where that is not the way out of the inside cell
        out_pos = a[kk, jj, ii]
        flip = out_pos != (axis != 1)
        t0 = np.where(flip[:, None], np.stack([q00, q11, q10], axis=1), np.stack([q00, q10, q11], axis=1))
        t1 = np.where(flip[:, None], np.stack([q00, q01, q11], axis=1), np.stack([q00, q11, q01], axis=1))
        out.append(np.stack([t0, t1], axis=1).reshape(-1, 3))
    return np.concatenate(out, axis=0).astype(np.int32)


def tile_order(width: int, height: int, tile_w: int = TILE_W, tile_h: int = TILE_H):
    """Pixel (px, py) of every ray index, in warp-tile order (see module doc)."""
    idx_px = np.empty(width * height, dtype=np.int64)
    idx_py = np.empty(width * height, dtype=np.int64)
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    ty, ly = py // tile_h, py % tile_h
    tx, lx = px // tile_w, px % tile_w
    th = np.minimum(tile_h, height - ty * tile_h)
    tw = np.minimum(tile_w, width - tx * tile_w)
    ray = ty * tile_h * width + tx * tile_w * th + ly * tw + lx
    idx_px[ray.ravel()] = px.ravel()
    idx_py[ray.ravel()] = py.ravel()
    return idx_px, idx_py


@dataclass(frozen=True)
class Camera:
    eye: tuple
    fov_deg: float
    width: int
    height: int

    def constants(self):
        """float32 constants of the pixel -> direction recipe (computed in float64, rounded once)."""
        short = min(self.width, self.height)
        tanh = math.tan(math.radians(self.fov_deg) * 0.5)
        f = np.float32
        return dict(kx=f(2.0 / self.width), ky=f(2.0 / self.height),
                    tx=f(tanh * (self.width / short)), ty=f(tanh * (self.height / short)))


def camera_rays(cam: Camera):
    """Origins and directions (float32 [W*H, 3]) in warp-tile order.

    Every operation below is one correctly rounded float32 operation, in this
    order (no fused multiply-add):
      sx = ((px + 0.5)*kx - 1)*tx ; sy = (1 - (py + 0.5)*ky)*ty ;
      s2 = (sx*sx + sy*sy) + 1 ; L = sqrt(s2) ; d = (sx/L, sy/L, 1/L)
    """
    c = cam.constants()
    f = np.float32
    px, py = tile_order(cam.width, cam.height)
    sx = ((px.astype(f) + f(0.5)) * c["kx"] - f(1.0)) * c["tx"]
    sy = (f(1.0) - (py.astype(f) + f(0.5)) * c["ky"]) * c["ty"]
    s2 = (sx * sx + sy * sy) + f(1.0)
    L = np.sqrt(s2)
    d = np.stack([sx / L, sy / L, f(1.0) / L], axis=1).astype(f)
    o = np.broadcast_to(np.asarray(cam.eye, dtype=f), d.shape).copy()
    return o, d


def interior_points(count: int, seed: int, lo: float = 0.05, hi: float = 0.95):
    return _rng(seed, 2).uniform(lo, hi, size=(count, 3)).astype(np.float32)


def uniform_directions(count: int, seed: int):
    """Unit vectors uniform on the sphere (float64 normalised, rounded to float32)."""
    g = _rng(seed, 3)
    z = g.uniform(-1.0, 1.0, size=count)
    phi = g.uniform(0.0, 2.0 * math.pi, size=count)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


@dataclass
class Scene:
    name: str
    n: int
    jitter: float
    seed: int
    points: np.ndarray
    tets: np.ndarray
    tris: np.ndarray
    inside: np.ndarray
    spheres: tuple = field(default=None)
    camera: Camera | None = None

    @property
    def n_tets(self):
        return int(self.tets.shape[0])

    @property
    def n_points(self):
        return int(self.points.shape[0])

    @property
    def n_tris(self):
        return int(self.tris.shape[0])


def make_grid_scene(name, n, jitter, seed, spheres=None, n_spheres=0, camera=None, inside=None):
    pts, tets = freudenthal_grid(n, jitter, seed)
    if inside is None:
        if spheres is None:
            spheres = random_spheres(n_spheres, seed)
        inside = inside_cells(n, *spheres)
    tris = constrained_faces(n, inside)
    return Scene(name, n, jitter, seed, pts, tets, tris, inside, spheres, camera)


# The five workloads.  Sizes, jitter, sphere counts, cameras and ray counts
# follow the workload table of the project; seeds are fixed here.
CONFIGS = {
    "tiny": dict(n=8, jitter=0.10, seed=1001,
                 spheres=(np.array([[0.5, 0.5, 0.5]]), np.array([0.3])),
                 camera=Camera((0.5, 0.5, 0.05), 60.0, 64, 64)),
    "medium": dict(n=64, jitter=0.15, seed=1002, n_spheres=16,
                   camera=Camera((0.5, 0.5, 0.02), 70.0, 1920, 1080)),
    "precision": dict(n=128, jitter=0.15, seed=1003, n_spheres=64,
                      camera=Camera((0.5, 0.5, 0.02), 70.0, 2048, 2048)),
    "large": dict(n=256, jitter=0.15, seed=1005, n_spheres=256,
                  camera=Camera((0.5, 0.5, 0.02), 70.0, 1024, 1024)),
}

# Per-config secondary-ray recipe: one cosine bounce per hit ("precision"),
# eight ambient-occlusion rays with t_max = 0.05 per hit ("large").
SECONDARY = {"precision": dict(kind="bounce", per_hit=1, tmax=float("inf")),
             "large": dict(kind="ao", per_hit=8, tmax=0.05)}

BATCHED = dict(n_meshes=32, grid_choices=(16, 24, 32, 48, 64, 96), spheres=(4, 32),
               rays=(1_000, 2_000_000), seed=1004, jitter=0.15,
               camera_eye=(0.5, 0.5, 0.02), fov_deg=70.0)


def make_config(name: str, n_override: int | None = None) -> Scene:
    cfg = dict(CONFIGS[name])
    n = n_override or cfg.pop("n")
    cfg.pop("n", None)
    return make_grid_scene(name, n, **cfg)


def batched_meshes(max_rays: int | None = None, scale: float = 1.0):
    """Descriptors of the 32-mesh uneven workload (grid n, sphere count, rays, primary share).

    Ray counts are log-uniform in [1e3, 2e6]; about half of each batch are
    primary camera rays and half uniform-direction rays from interior points.
    `scale` shrinks every ray count (for small test runs).
    """
    g = _rng(BATCHED["seed"], 4)
    out = []
    for m in range(BATCHED["n_meshes"]):
        n = int(g.choice(BATCHED["grid_choices"]))
        k = int(g.integers(BATCHED["spheres"][0], BATCHED["spheres"][1] + 1))
        lo, hi = math.log(BATCHED["rays"][0]), math.log(BATCHED["rays"][1])
        rays = int(round(math.exp(g.uniform(lo, hi)) * scale))
        rays = max(rays, 1)
        if max_rays is not None:
            rays = min(rays, max_rays)
        out.append(dict(mesh=m, n=n, n_spheres=k, rays=rays, seed=BATCHED["seed"] * 100 + m,
                        primary=rays // 2))
    return out
