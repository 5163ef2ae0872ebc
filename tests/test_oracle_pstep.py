"""Pins of the oracle's per-fragment pixel step (pstep, Sec. 1.1.1): each
distance's ramp is its own fwidth, |d_i g| + |d_j g|, with d g = n . d G
from the map's central differences.
  * A straight edge of a narrow pinhole view: the ramp at a pixel is the
    textbook fwidth anti-aliasing of a straight line, clamp(d / (|cos phi| +
    |sin phi|) + 1/2) with d the pixel's distance to the projected line in
    pixels and phi the line normal's angle in the image (the L1 footprint
    of fwidth).
  * A closed icosphere: shared edges have opposite normals, hence equal
    widths and complementary ramps: coverage 1 away from the vertices and
    one centre-inside triangle per pixel.
  * 8x8 supersampling: per-triangle sums within 1 %."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@pytest.mark.parametrize("phi_deg", [0.0, 20.0, 45.0, 71.0])
def test_straight_edge_ramp_is_fwidth_antialiasing(phi_deg):
    W = H = 96
    omega = 8.0  # narrow: the map is nearly affine over the picture
    m, dm = oracle.make_map_spec(W, H, oracle.MAP_RECTILINEAR, (omega,), derivs=True)
    # image plane z = cot(omega/2) (x, y the view coordinates, x = 2 f_s - 1);
    # a line through the picture centre offset by c, normal (cos phi, sin phi)
    f = 1 / np.tan(np.radians(omega / 2))
    phi = np.radians(phi_deg)
    nrm = np.array([np.cos(phi), np.sin(phi)])
    c = 0.013
    # a triangle with that line as its first edge, far corners off-picture
    tv = np.array([-nrm[1], nrm[0]])
    p0 = c * nrm - 3 * tv
    p1 = c * nrm + 3 * tv
    p2 = c * nrm + 3 * nrm  # on the positive side
    tri = np.array([[[p[0], p[1], f] for p in (p0, p1, p2)]]) * 5.0
    r = oracle.raster_pstep(m, dm, oracle.setup64(tri))
    i, j = np.meshgrid(np.arange(W), np.arange(H))
    x = (2 * i + 1) / W - 1
    y = ((2 * j + 1) / H - 1) / (W / H)
    d = (x * nrm[0] + y * nrm[1] - c) / (2 / W)  # signed distance in pixels
    expect = np.clip(d / (abs(np.cos(phi)) + abs(np.sin(phi))) + 0.5, 0, 1)
    near = np.abs(d) < 3  # the ramp, away from the far corners
    assert np.abs(r["cov"][near] - expect[near]).max() < 2e-3


def test_icosphere_pstep_is_watertight():
    W, H = 80, 60
    m, dm = oracle.make_map_spec(W, H, oracle.MAP_UNIVERSAL, oracle.limits(0.3, 0.8, 0.9, 250.0), derivs=True)
    tris = scenes.icosphere(2, 50.0)
    r = oracle.raster_pstep(m, dm, oracle.setup(tris), extras=True)
    valid = m[..., 3] > 0
    assert np.all(r["n_inside"][valid] == 1)
    V = _unit(np.unique(tris.reshape(-1, 3).astype(np.float64), axis=0))
    near_vertex = np.arccos(np.clip((m[..., :3] @ V.T).max(-1), -1, 1)) * m[..., 3] < 2.0
    ok = valid & ~near_vertex
    assert np.abs(r["cov"][ok] - 1).max() < 1e-9


def test_pstep_supersampling_agreement():
    W = H = 64
    lens = (0.0, 1.0, 1.0, 180.0)
    m, dm = oracle.make_map_spec(W, H, oracle.MAP_UNIVERSAL, lens, derivs=True)
    tris = scenes.random_triangles(8, 3.0, 8.0, 0.9, seed=31)
    ss = 8
    off = (np.arange(ss) + 0.5) / ss - 0.5
    i, j = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    fs = (i[..., None, None] + 0.5 + off[None, None, None, :]) / W
    ft = (j[..., None, None] + 0.5 + off[None, None, :, None]) / H
    fs, ft = np.broadcast_arrays(fs, ft)
    sub, sub_ok = oracle.map_dirs(fs.copy(), ft.copy(), W, H, lens)
    n_big = 0
    for t in range(len(tris)):
        out = oracle.raster_pstep(m, dm, oracle.setup(tris[t:t + 1]))
        coef = np.linalg.solve(tris[t].astype(np.float64).T, sub.reshape(-1, 3).T).T
        inside = (coef >= 0).all(1).reshape(H, W, ss, ss) & sub_ok
        frac = inside.mean(axis=(2, 3))
        if frac.sum() >= 100:
            n_big += 1
            assert abs(out["cov"].sum() / frac.sum() - 1) < 0.01, (t, out["cov"].sum(), frac.sum())
    assert n_big >= 1
