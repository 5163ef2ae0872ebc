"""Pins of the oracle's other perspective maps (Sec. 2.2) and of the lens
distortion of view coordinates (Sec. 2.3), each against something other
than its own formula:
  * the rectilinear map against the Universal model at k = 1 (pinned to the
    textbook gnomonic law in test_oracle_map), for every AOV type;
  * the solid angle each map covers, integrated from its Jacobian, against
    closed forms: the whole sphere (equirectangular, cube), a cylindrical
    band (curved panorama), a spherical cap (full dome);
  * a closed icosphere around the eye rasterized through each map covers
    every valid pixel exactly once (the maps are continuous and injective
    away from their charts' borders);
  * Brown-Conrady radial distortion composed with the pinhole and the
    equidistant laws;
  * the cube's front face equals a 90-degree square rectilinear view."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes


@pytest.mark.parametrize("aov", [0, 1, 2, 3])
def test_rectilinear_equals_universal_k1(aov):
    for omega in (40.0, 90.0, 150.0):
        r = oracle.make_map_spec(64, 40, oracle.MAP_RECTILINEAR, (omega,), aov=aov)
        u, _ = oracle.make_map(64, 40, 1.0, 1.0, 1.0, omega, aov=aov)
        assert np.abs(r - u).max() < 1e-12 * max(1.0, np.abs(u[..., 3]).max())


def _solid_angle(kind, param, W, H, n_s, n_t, s_range=(0.0, 1.0), t_range=(0.0, 1.0)):
    # midpoint rule over texture coordinates, |v . (dv/ds x dv/dt)| by central
    # differences of the map function (h = 1e-6)
    s = s_range[0] + (np.arange(n_s) + 0.5) / n_s * (s_range[1] - s_range[0])
    t = t_range[0] + (np.arange(n_t) + 0.5) / n_t * (t_range[1] - t_range[0])
    S, T = np.meshgrid(s, t)
    S, T = S.ravel(), T.ravel()
    h = 1e-6
    v0, ok = oracle.map_spec_dirs(S, T, W, H, kind, param)
    vsp, _ = oracle.map_spec_dirs(S + h, T, W, H, kind, param)
    vsm, _ = oracle.map_spec_dirs(S - h, T, W, H, kind, param)
    vtp, _ = oracle.map_spec_dirs(S, T + h, W, H, kind, param)
    vtm, _ = oracle.map_spec_dirs(S, T - h, W, H, kind, param)
    ds = (vsp - vsm) / (2 * h)
    dt = (vtp - vtm) / (2 * h)
    jac = np.abs(np.einsum("ij,ij->i", v0, np.cross(ds, dt)))
    da = (s_range[1] - s_range[0]) / n_s * (t_range[1] - t_range[0]) / n_t
    return float(np.sum(jac[ok]) * da)


def test_solid_angles_against_closed_forms():
    four_pi = 4 * np.pi
    assert abs(_solid_angle(oracle.MAP_EQUIRECT, (), 64, 32, 400, 200) / four_pi - 1) < 1e-4
    # the cube: each face separately (the chart changes at face borders)
    total = sum(_solid_angle(oracle.MAP_CUBE, (), 60, 10, 120, 120, (f / 6 + 1e-9, (f + 1) / 6 - 1e-9))
                for f in range(6))
    assert abs(total / four_pi - 1) < 1e-4
    # curved panorama: a band of a unit cylinder, Omega_h wide and `height`
    # tall, seen from the axis: Omega_h * 2 sin(atan(height / 2))
    om, hh = 200.0, 1.5
    exact = np.radians(om) * hh / np.sqrt(1 + hh * hh / 4)
    assert abs(_solid_angle(oracle.MAP_PANORAMA, (om, hh), 64, 32, 300, 300) / exact - 1) < 1e-4


def test_dome_solid_angle_is_a_cap():
    # the dome disk in polar coordinates (exact boundary): theta_max =
    # compression + 90 deg, solid angle 2 pi (1 - cos theta_max)
    comp = 30.0
    n_r, n_p = 300, 600
    r = (np.arange(n_r) + 0.5) / n_r
    ph = (np.arange(n_p) + 0.5) / n_p * 2 * np.pi
    R, P = np.meshgrid(r, ph)
    R, P = R.ravel(), P.ravel()

    def dirs(RR, PP):
        fs = (1 + RR * np.cos(PP)) / 2
        ft = (1 - RR * np.sin(PP)) / 2
        v, ok = oracle.map_spec_dirs(fs, ft, 64, 64, oracle.MAP_DOME, (comp, 0.0, 0.0))
        return v

    h = 1e-6
    v0 = dirs(R, P)
    dr = (dirs(R + h, P) - dirs(R - h, P)) / (2 * h)
    dp = (dirs(R, P + h) - dirs(R, P - h)) / (2 * h)
    total = np.sum(np.abs(np.einsum("ij,ij->i", v0, np.cross(dr, dp)))) / n_r * (2 * np.pi / n_p)
    exact = 2 * np.pi * (1 - np.cos(np.radians(comp + 90)))
    assert abs(total / exact - 1) < 1e-4


@pytest.mark.parametrize("kind,param,W,H", [
    (oracle.MAP_EQUIRECT, (), 96, 48),
    (oracle.MAP_CUBE, (), 96, 16),
    (oracle.MAP_PANORAMA, (300.0, 1.2), 96, 40),
    (oracle.MAP_DOME, (40.0, 20.0, 0.0), 64, 64),
])
def test_watertight_icosphere_through_each_map(kind, param, W, H):
    m = oracle.make_map_spec(W, H, kind, param)
    tris = scenes.icosphere(2, 50.0)
    r = oracle.raster(m, oracle.setup(tris), extras=True)
    valid = m[..., 3] > 0
    assert valid.sum() > 0.5 * W * H
    assert np.all(r["n_inside"][valid] == 1)
    assert np.all(r["n_inside"][~valid] == 0)


def test_brown_conrady_radial_laws():
    # pinhole: tan(theta) = tan(Omega/2) r (1 + k1 r^2 + k2 r^4); equidistant
    # (Universal k = 0): theta = (Omega/2) r (1 + k1 r^2 + k2 r^4)
    W, H = 64, 48
    k1, k2 = -0.12, 0.03
    fs = (np.arange(W) + 0.5) / W
    ft = (np.arange(H) + 0.5) / H
    FS, FT = np.meshgrid(fs, ft)
    x = 2 * FS - 1
    y = (2 * FT - 1) / (W / H)
    r = np.hypot(x, y)
    rd = r * (1 + k1 * r ** 2 + k2 * r ** 4)
    m = oracle.make_map_spec(W, H, oracle.MAP_RECTILINEAR, (100.0,), dist=(k1, k2))
    theta = np.arccos(np.clip(m[..., 2], -1, 1))
    assert np.abs(np.tan(theta) - np.tan(np.radians(50.0)) * rd).max() < 1e-12
    m = oracle.make_map_spec(W, H, oracle.MAP_UNIVERSAL, (0.0, 1.0, 1.0, 160.0), dist=(k1, k2))
    theta = np.arccos(np.clip(m[..., 2], -1, 1))
    assert np.abs(theta - np.radians(80.0) * rd).max() < 1e-12
    # no distortion: the plain map
    u, _ = oracle.make_map(W, H, 0.3, 0.8, 0.9, 200.0)
    d = oracle.make_map_spec(W, H, oracle.MAP_UNIVERSAL, (0.3, 0.8, 0.9, 200.0))
    assert np.array_equal(u, d)


def test_cube_front_face_is_a_square_rectilinear_view():
    F = 24
    c = oracle.make_map_spec(6 * F, F, oracle.MAP_CUBE)
    front = c[:, 3 * F:4 * F, :3]
    r = oracle.make_map_spec(F, F, oracle.MAP_RECTILINEAR, (90.0,))
    assert np.abs(front - r[..., :3]).max() < 1e-12
