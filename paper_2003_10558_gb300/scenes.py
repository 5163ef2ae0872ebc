"""Seeded synthetic inputs: triangle scenes, icospheres, cameras, lens draws.

This module holds input generation only -- none of the rasterizer's
arithmetic -- so that the CUDA path and the FP64 oracle can be fed the same
arrays.  All geometry is generated in float64 with numpy's seeded PCG64
generator and rounded to float32 once.

Scene recipe (the paper measures on no dataset; these stand in for the
"randomly placed small triangles around the eye" workloads):
  * centroid direction uniform on the sphere: z ~ U[-1, 1], phi ~ U[0, 2 pi);
  * one radius rho ~ U[rho_min, rho_max] per triangle;
  * tangent basis (t1, t2) at the centroid direction c: t1 = normalize(c x e)
    with e the x axis (y axis when c is within 0.9 of x), t2 = c x t1;
  * each vertex = rho * expmap(c, u t1 + v t2), u, v ~ U[-j, j] rad, so the
    mean edge length is about 1.04 j.
"""
from __future__ import annotations

import numpy as np

VIEW_SIZES = ((512, 512), (1024, 1024), (2048, 1024), (1920, 1080))


def _unit_sphere(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _tangent_basis(c):
    e = np.zeros_like(c)
    near_x = np.abs(c[:, 0]) > 0.9
    e[~near_x, 0] = 1.0
    e[near_x, 1] = 1.0
    t1 = np.cross(c, e)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(c, t1)
    return t1, t2


def random_triangles(n, rho_min, rho_max, jitter, seed):
    """[n, 3, 3] float32 world-space triangles around the origin."""
    rng = np.random.default_rng(seed)
    c = _unit_sphere(rng, n)
    rho = rng.uniform(rho_min, rho_max, n)
    uv = rng.uniform(-jitter, jitter, (n, 3, 2))
    t1, t2 = _tangent_basis(c)
    w = uv[..., 0:1] * t1[:, None, :] + uv[..., 1:2] * t2[:, None, :]
    ang = np.linalg.norm(w, axis=2, keepdims=True)
    safe = np.where(ang > 0.0, ang, 1.0)
    d = np.cos(ang) * c[:, None, :] + np.sin(ang) * w / safe
    return (rho[:, None, None] * d).astype(np.float32)


def icosphere(level, radius):
    """[20*4^level, 3, 3] float32 triangles of a subdivided icosahedron of the
    given radius around the origin.  Vertices are shared bitwise between
    neighbouring triangles and every face is wound the same way (outward)."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
             (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = (np.array(verts) * radius).astype(np.float32)
    F = np.array(faces, dtype=np.int64)
    return V[F]


def camera(origin=(0.0, 0.0, 0.0), M=None):
    """12 float32: eye position O then the 3x3 world->camera rotation M
    (row-major); camera-space X' = M (X - O)."""
    if M is None:
        M = np.eye(3)
    return np.concatenate([np.asarray(origin, dtype=np.float64).ravel(),
                           np.asarray(M, dtype=np.float64).ravel()]).astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads.

def tiny_scene(seed=0):
    """256x256 equidistant view (k=0, l=1, s=1, Omega=180 deg) of 64
    triangles, rho ~ U[1, 10], jitter 0.25 rad."""
    lens = dict(W=256, H=256, k=0.0, l=1.0, s=1.0, omega=180.0)
    return lens, random_triangles(64, 1.0, 10.0, 0.25, seed), camera()


def single_view_scene(seed=1, n_random=200_000):
    """1920x1080 view (k=0.32, l=0.62, s=0.86, Omega=270 deg) of a level-5
    icosphere of radius 50 around the eye (20,480 triangles) plus n_random
    triangles with rho ~ U[1, 40] and edge ~0.02 rad (jitter 0.0192)."""
    lens = dict(W=1920, H=1080, k=0.32, l=0.62, s=0.86, omega=270.0)
    tris = np.concatenate([icosphere(5, 50.0), random_triangles(n_random, 1.0, 40.0, 0.0192, seed)])
    return lens, tris, camera()


def batched_views(n_views=64, seed=2):
    """Per-view lens and camera draws: size uniform over VIEW_SIZES,
    k ~ U[-1, 1], l, s ~ U[0.5, 1], Omega ~ U[90, 360] deg, eye uniform in a
    ball of radius 5."""
    rng = np.random.default_rng(seed)
    views = []
    for _ in range(n_views):
        W, H = VIEW_SIZES[rng.integers(len(VIEW_SIZES))]
        k = rng.uniform(-1.0, 1.0)
        l = rng.uniform(0.5, 1.0)
        s = rng.uniform(0.5, 1.0)
        om = rng.uniform(90.0, 360.0)
        d = _unit_sphere(rng, 1)[0]
        r = 5.0 * rng.uniform() ** (1.0 / 3.0)
        views.append(dict(W=int(W), H=int(H), k=float(k), l=float(l), s=float(s), omega=float(om),
                          cam=camera(r * d)))
    return views


def batched_scene(seed=2, n=1_000_000):
    """Shared scene of the batched workload: rho ~ U[1, 60], edge ~0.01 rad."""
    return random_triangles(n, 1.0, 60.0, 0.0096, seed)


# Differentiation workload: 1024 x 1024, 10,000 triangles of the tiny-scene
# generator with rho ~ U[1, 10] and jitter 0.05 rad (depth complexity about
# one over the sphere), colours c_t ~ U[0.2, 1]; the target lens is
# (k, l, s) = (0.2, 0.7, 0.9), the fit starts from (0.6, 1, 1) with vertex
# noise N(0, 0.01^2) per coordinate.  Omega = 180 deg, horizontal AOV.
GRAD_TARGET = {"k": 0.2, "l": 0.7, "s": 0.9, "omega": 180.0}
GRAD_START = {"k": 0.6, "l": 1.0, "s": 1.0, "omega": 180.0}


def grad_scene(seed=4, n=10_000, W=1024, H=1024):
    """Returns (target lens, start lens, true tris, noisy tris, colours, W, H);
    triangles float32 [n, 3, 3], colours float32 [n]."""
    tris = random_triangles(n, 1.0, 10.0, 0.05, seed)
    rng = np.random.default_rng(seed + 1000)
    colors = rng.uniform(0.2, 1.0, n).astype(np.float32)
    noisy = (tris.astype(np.float64) + rng.normal(0.0, 0.01, tris.shape)).astype(np.float32)
    target = dict(GRAD_TARGET, W=W, H=H)
    start = dict(GRAD_START, W=W, H=H)
    return target, start, tris, noisy, colors, W, H
