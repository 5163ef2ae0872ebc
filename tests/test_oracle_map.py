"""Pins of the oracle's perspective map (Universal perspective 2D->3D, its
limits, the AOV normalisation and the global delta) against closed forms,
textbook projections and invariants -- nothing here re-types the oracle."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def test_limits_table():
    for row in _golden_rows("limits.txt"):
        lhs, rhs = row.split("|")
        k, l, s, om, strict = (float(v) for v in lhs.split())
        exp = [float(v) for v in rhs.split()]
        got = oracle.limits(k, l, s, om, strict=bool(strict))
        assert np.allclose(got, exp, atol=1e-12), (row, got)


# textbook theta(rho) with f fixed by rho(Omega/2) = 1
def _theta_textbook(name, rho, half):
    if name == "gnomonic":
        return np.arctan(np.tan(half) * rho)
    if name == "stereographic":
        return 2.0 * np.arctan(np.tan(half / 2.0) * rho)
    if name == "equidistant":
        return half * rho
    if name == "equisolid":
        return 2.0 * np.arcsin(np.clip(np.sin(half / 2.0) * rho, -1, 1))
    if name == "orthographic":
        return np.arcsin(np.clip(np.sin(half) * rho, -1, 1))
    raise KeyError(name)


@pytest.mark.parametrize("omega", [60.0, 120.0, 170.0])
def test_named_projections(omega):
    rows = [r.split() for r in _golden_rows("projections.txt")]
    rng = np.random.default_rng(5)
    xy = rng.uniform(-1.0, 1.0, (200, 2)) * 0.99
    xy[0] = (1e-9, 0.0)
    for r in rows:
        k, name = float(r[0]), r[1]
        eff = oracle.limits(k, 1.0, 1.0, omega)
        half = math.radians(eff[3]) / 2.0
        for x, y in xy:
            rho = math.hypot(x, y)
            th = _theta_textbook(name, rho, half)
            if name in ("equisolid", "orthographic") and rho * math.sin(half / (2 if name == "equisolid" else 1)) > 1:
                continue
            exp = np.array([x / rho * math.sin(th), y / rho * math.sin(th), math.cos(th)])
            v, ok = oracle.map_dir(x, y, eff)
            assert ok
            assert np.abs(v - exp).max() < 1e-12, (name, x, y, v, exp)


def test_gnomonic_is_rectilinear_map():
    """k = 1 reproduces the paper's rectilinear (pinhole) map
    normalize(2 f_s - 1, (2 f_t - 1)/a, cot(Omega/2)) (Sec. "Rectilinear
    perspective map")."""
    W, H, om = 64, 48, 100.0
    m, eff = oracle.make_map(W, H, 1.0, 1.0, 1.0, om)
    i, j = np.meshgrid(np.arange(W), np.arange(H))
    a = W / H
    w = np.stack([2 * (i + 0.5) / W - 1, (2 * (j + 0.5) / H - 1) / a,
                  np.full(i.shape, 1.0 / math.tan(math.radians(om) / 2))], -1)
    w /= np.linalg.norm(w, axis=-1, keepdims=True)
    assert np.abs(m[..., :3] - w).max() < 1e-13


def test_aov_normalisation():
    # horizontal: x in [-1, 1], y in [-1/a, 1/a]
    assert np.allclose(oracle.view_coord(1.0, 0.5, 16 / 9, 0), (1.0, 0.0))
    assert np.allclose(oracle.view_coord(0.5, 1.0, 16 / 9, 0), (0.0, 9 / 16))
    # vertical: y in [-1, 1]
    assert np.allclose(oracle.view_coord(0.5, 1.0, 16 / 9, 2), (0.0, 1.0))
    assert np.allclose(oracle.view_coord(1.0, 0.5, 16 / 9, 2), (16 / 9, 0.0))
    # diagonal: the corner is at unit distance
    x, y = oracle.view_coord(1.0, 1.0, 16 / 9, 1)
    assert abs(math.hypot(x, y) - 1.0) < 1e-15
    # horizontal 4x3: a 4:3 picture spans x in [-1, 1]
    assert np.allclose(oracle.view_coord(1.0, 0.5, 4 / 3, 3), (1.0, 0.0))


@pytest.mark.parametrize("k,l,s", [(0.32, 1.0, 0.86), (0.32, 0.62, 1.0), (-0.5, 0.7, 1.0), (0.0, 0.5, 1.0),
                                   (0.8, 0.9, 1.0), (-0.9, 1.0, 0.8)])
def test_round_trip_3d_to_2d(k, l, s):
    """The 3D->2D transform is the reverse of 2D->3D (Sec. "Transformation of
    3D->2D"); exactly so when s = 1 or l = 1 (see the anamorphic reading)."""
    eff = oracle.limits(k, l, s, 150.0)
    rng = np.random.default_rng(7)
    n = 0
    for x, y in rng.uniform(-1, 1, (300, 2)):
        v, ok = oracle.map_dir(x, y, eff)
        if not ok or v[2] < -0.99:
            continue
        x2, y2 = oracle.map_inverse(v, eff)
        assert abs(x2 - x) < 1e-12 and abs(y2 - y) < 1e-12, (x, y, x2, y2)
        n += 1
    assert n > 100


def test_map_invariants():
    W, H = 96, 64
    for k, l, s, om in [(0.32, 0.62, 0.86, 270.0), (-1.0, 1.0, 1.0, 180.0), (0.0, 0.7, 0.9, 360.0),
                        (1.0, 1.0, 1.0, 150.0)]:
        m, eff = oracle.make_map(W, H, k, l, s, om)
        valid = m[..., 3] > 0
        assert valid.any()
        # invalid pixels are all zero
        assert np.all(m[~valid] == 0.0)
        # unit directions
        assert np.abs(np.linalg.norm(m[valid][:, :3], axis=1) - 1).max() < 1e-14
        # mirror symmetry about the vertical axis: v(-x, y) = (-v_x, v_y, v_z)
        mir = m[:, ::-1]
        assert np.abs(mir[..., 0] + m[..., 0]).max() < 1e-14
        assert np.abs(mir[..., 1:4] - m[..., 1:4]).max() < 1e-9 * max(1.0, m[..., 3].max())
        # and about the horizontal axis
        flp = m[::-1]
        assert np.abs(flp[..., 1] + m[..., 1]).max() < 1e-14


def test_orthographic_invalid_corners():
    """k = -1, Omega = 180: asin(sin(-pi/2) R) is undefined for R > 1, i.e. in
    the corners of a square picture; those pixels are invalid (zero)."""
    W = H = 64
    m, _ = oracle.make_map(W, H, -1.0, 1.0, 1.0, 180.0)
    i, j = np.meshgrid(np.arange(W), np.arange(H))
    R = np.hypot(2 * (i + 0.5) / W - 1, 2 * (j + 0.5) / H - 1)
    assert np.array_equal(m[..., 3] > 0, R <= 1.0)


@pytest.mark.parametrize("W,om", [(256, 180.0), (512, 90.0), (1024, 270.0)])
def test_delta_closed_form_equidistant(W, om):
    """Equidistant (k = 0, l = s = 1): near the image centre one pixel step
    turns the direction by Omega/W radians, almost all of it in the x
    component, so the global delta is W/Omega (Sec. 1.1.1, global delta)."""
    m, _ = oracle.make_map(W, W, 0.0, 1.0, 1.0, om)
    c = W // 2
    exp = W / math.radians(om)
    assert abs(m[c, c, 3] / exp - 1.0) < 2e-4
    assert abs(m[c - 1, c - 1, 3] / exp - 1.0) < 2e-4


def test_delta_orthographic_row():
    """Orthographic, Omega = 180 (k = -1): on the centre row v_x = x and
    v_z = sqrt(1 - x^2), so one pixel step (dx = 2/W) changes v_x by 2/W and
    v_z by (2/W)|x|/sqrt(1 - x^2); delta is the reciprocal of the larger.
    Next to undefined pixels the derivative falls back to one side, so every
    valid pixel keeps a finite positive delta."""
    W = 256
    m, _ = oracle.make_map(W, W, -1.0, 1.0, 1.0, 180.0)
    d = m[..., 3]
    valid = d > 0
    assert np.isfinite(d[valid]).all() and (d[valid] > 0).all()
    j = W // 2
    for i in range(W):
        x = 2 * (i + 0.5) / W - 1
        if abs(x) > 0.9:
            continue
        exp = (W / 2) / max(1.0, abs(x) / math.sqrt(1 - x * x))
        assert abs(d[j, i] / exp - 1) < 1e-2, (i, d[j, i], exp)
