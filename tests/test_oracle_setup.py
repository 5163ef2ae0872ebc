"""Pins of the oracle's triangle set-up: edge-plane normals (Sec. 1.1), the
miter smallest circle (Sec. 1.1.2) against a brute-force smallest enclosing
cap, the plane depth (Sec. 1.1.4) against a closed form, and culling."""
import itertools

import numpy as np

import oracle
from paper_2003_10558_gb300 import scenes


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_edge_normals_perpendicular_and_oriented():
    tris = scenes.random_triangles(500, 1.0, 10.0, 0.25, seed=11)
    rec = oracle.setup(tris)
    assert (rec[:, oracle.REC_VALID] == 1).all()
    V = tris.astype(np.float64)
    cen = _unit(V.sum(1))
    for e, (p, q) in enumerate([(0, 1), (1, 2), (2, 0)]):
        n = rec[:, 3 * e:3 * e + 3]
        assert np.abs(np.linalg.norm(n, axis=1) - 1).max() < 1e-14
        for w in (p, q):
            assert np.abs((n * _unit(V[:, w])).sum(1)).max() < 1e-13
        # the third vertex and the centroid direction are on the inside
        other = 3 - p - q
        assert ((n * V[:, other]).sum(1) > 0).all()
        assert ((n * cen).sum(1) > 0).all()


def test_shared_edges_have_opposite_normals_bitwise():
    tris = scenes.icosphere(2, 50.0)
    rec = oracle.setup(tris)
    edges = {}
    for t in range(len(tris)):
        for e, (p, q) in enumerate([(0, 1), (1, 2), (2, 0)]):
            a, b = tris[t, p].tobytes(), tris[t, q].tobytes()
            edges.setdefault(frozenset((a, b)), []).append(rec[t, 3 * e:3 * e + 3])
    assert len(edges) == 3 * len(tris) // 2
    for ns in edges.values():
        assert len(ns) == 2
        assert np.array_equal(ns[0], -ns[1])


def _brute_smallest_cap(U):
    """Smallest spherical cap (centre, cos radius) holding three unit vectors:
    every pair-diameter cap and the circumscribed cap, keep the smallest that
    holds all three."""
    cands = []
    for a, b in itertools.combinations(range(3), 2):
        c = _unit(U[a] + U[b])
        cands.append((c, float(c @ U[a])))
    nrm = np.cross(U[1] - U[0], U[2] - U[0])
    c = _unit(nrm)
    if c @ U[0] < 0:
        c = -c
    cands.append((c, float(c @ U[0])))
    best = None
    for c, cosr in cands:
        if all(c @ u >= cosr - 1e-12 for u in U) and (best is None or cosr > best[1]):
            best = (c, cosr)
    return best


def test_miter_is_smallest_enclosing_cap():
    tris = np.concatenate([scenes.random_triangles(400, 1.0, 10.0, 0.25, seed=3),
                           scenes.random_triangles(400, 1.0, 10.0, 1.2, seed=4)])
    rec = oracle.setup(tris)
    n_obtuse = 0
    for t in range(len(tris)):
        U = _unit(tris[t].astype(np.float64))
        c, cosr = _brute_smallest_cap(U)
        S = rec[t, oracle.REC_S:oracle.REC_S + 3]
        assert np.abs(S - c).max() < 1e-9, t
        assert abs(rec[t, oracle.REC_C] - cosr) < 1e-12, t
        on_rim = np.abs(U @ S - rec[t, oracle.REC_C]) < 1e-12
        assert on_rim.sum() >= 2
        n_obtuse += on_rim.sum() == 2
    # both branches of the construction were exercised
    assert 50 < n_obtuse < len(tris) - 50


def test_plane_depth_closed_form():
    """A triangle in the plane z = D is at distance r = D / G_z along G."""
    D = 7.5
    tris = np.array([[[-20, -20, D], [30, -20, D], [0, 30, D]]], dtype=np.float32)
    m, _ = oracle.make_map(48, 48, 0.0, 1.0, 1.0, 120.0)
    rec = oracle.setup(tris)
    out = oracle.raster(m, rec)
    hit = out["id"] == 0
    assert hit.sum() > 500
    exp = D / m[..., 2]
    assert np.abs(out["depth"][hit] / exp[hit] - 1).max() < 1e-13
    assert np.isinf(out["depth"][~hit]).all()


def test_culling():
    tris = np.array([
        [[0, 0, 0], [1, 0, 5], [0, 1, 5]],      # vertex at the eye
        [[1, 0, 1], [2, 0, 2], [0, 1, 3]],      # A, B collinear with O: A'.(B' x C') = 0
        [[1, 0, 5], [0, 1, 5], [-1, -1, 5]],    # ordinary
    ], dtype=np.float32)
    rec = oracle.setup(tris)
    assert list(rec[:, oracle.REC_VALID]) == [0.0, 0.0, 1.0]


def test_camera_transform():
    """Moving the eye and rotating the camera is the same as moving the scene
    the opposite way: X' = M (X - O)."""
    tris = scenes.random_triangles(50, 2.0, 9.0, 0.3, seed=9)
    O = np.array([0.5, -1.0, 2.0])
    th = 0.7
    M = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    rec_cam = oracle.setup(tris, scenes.camera(O, M))
    cam32 = scenes.camera(O, M)
    moved = np.einsum("ij,tvj->tvi", cam32[3:].astype(np.float64).reshape(3, 3),
                      tris.astype(np.float64) - cam32[:3].astype(np.float64))
    rec_ref = oracle.setup(moved.astype(np.float32))
    ok = (rec_cam[:, oracle.REC_VALID] == 1) & (rec_ref[:, oracle.REC_VALID] == 1)
    assert ok.sum() > 40
    assert np.abs(rec_cam[ok, :12] - rec_ref[ok, :12]).max() < 1e-6
