"""Pins of the oracle's gradient of the shaded image (the differentiable
workload): its analytic FP64 adjoint against FP64 central finite
differences of its own forward (h = 1e-6, vertices in float64 so the step is
exact), the complex-step map tangents against central differences of the
map, and the two homogeneity identities of a render seen from the origin:
the image depends on vertex directions only (degree 0 in the vertices, so
sum V . dL/dV = 0) and the depth is degree 1 (sum V . d depth/dV = depth)."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

LIMITS_HI = {"k": 1.0, "l": 1.0, "s": 1.0}


def _fd_lens(lens, name, f, h=1e-6):
    """Central difference, one-sided from inside the domain at an upper
    parameter limit (the gradient there is the one of the clamped map)."""
    lp, lm = dict(lens), dict(lens)
    if name in LIMITS_HI and lens[name] + h > LIMITS_HI[name]:
        lm2 = dict(lens)
        lm[name] -= h
        lm2[name] -= 2 * h
        return (3 * f(lens) - 4 * f(lm) + f(lm2)) / (2 * h)
    lp[name] += h
    lm[name] -= h
    return (f(lp) - f(lm)) / (2 * h)


@pytest.mark.parametrize("lens", [
    {"k": 0.4, "l": 0.8, "s": 0.9, "omega": 200.0},
    {"k": 0.0, "l": 0.6, "s": 0.7, "omega": 150.0},
    {"k": -0.5, "l": 0.9, "s": 0.8, "omega": 170.0},
])
def test_map_tangent_matches_central_differences(lens):
    W, H = 40, 30
    eff = oracle.limits(lens["k"], lens["l"], lens["s"], lens["omega"])
    names = ["k", "l", "s", "omega"]
    for j, name in enumerate(names):
        tan = oracle.map_tangent(W, H, eff, j)
        h = 1e-6
        lp, lm = dict(lens), dict(lens)
        lp[name] += h
        lm[name] -= h
        mp, _ = oracle.make_map(W, H, lp["k"], lp["l"], lp["s"], lp["omega"])
        mm, _ = oracle.make_map(W, H, lm["k"], lm["l"], lm["s"], lm["omega"])
        ok = (mp[..., 3] > 0) & (mm[..., 3] > 0)
        fd = (mp - mm) / (2 * h)
        # directions are O(1): absolute error against max(scale, 1); at k = 0 the
        # map is flat in k (the two branches agree to second order), where the
        # central difference itself is O(h)
        scale = np.maximum(np.abs(fd[ok]).max(axis=0), 1.0)
        scale[3] = max(scale[3], mp[ok][:, 3].max())  # delta: relative to its own size
        err = np.abs(tan[ok] - fd[ok]) / scale
        assert err[:, :3].max() < 1e-6, (name, err[:, :3].max())
        # delta is a max over components: allow the rare pixel at a switch
        assert np.mean(err[:, 3] < 1e-5) > 0.999, (name, np.sort(err[:, 3])[-5:])


def _small_case(seed=7, T=12, W=48, H=48):
    tris = scenes.random_triangles(T, 1.0, 3.0, 0.3, seed=seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    cols = rng.uniform(0.2, 1.0, T)
    return tris, cols, W, H, rng


@pytest.mark.parametrize("lens", [
    {"k": 0.4, "l": 0.8, "s": 0.9, "omega": 200.0},
    {"k": -0.3, "l": 0.7, "s": 0.85, "omega": 160.0},
    {"k": 1.0, "l": 1.0, "s": 1.0, "omega": 100.0},
])
def test_shade_gradient_matches_finite_differences(lens):
    tris, cols, W, H, rng = _small_case()
    m, eff = oracle.make_map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
    pix = np.arange(W * H)
    wts = rng.normal(size=W * H)
    g = oracle.render_grad(m, eff, tris, cols, wts, pixels=pix)
    idx = [(t, v, c) for t in range(tris.shape[0]) for v in range(3) for c in range(3)]
    fd = oracle.shade_fd(tris, cols, lens, pix, W, H, which=(), vert_idx=idx, weights=wts)

    def total(ln):
        mm, _ = oracle.make_map(W, H, ln["k"], ln["l"], ln["s"], ln["omega"])
        return float(np.sum(wts * oracle.shade(mm, oracle.setup64(tris), cols, pix)))

    gl = np.array([_fd_lens(lens, n, total) for n in ("k", "l", "s", "omega")])
    scale = np.abs(gl).max()
    assert np.all(np.abs(g["dlens"] - gl) <= 1e-4 * scale + 1e-3 * np.abs(gl)), (g["dlens"], gl)
    a = np.array([g["dtris"][i] for i in idx])
    b = np.array([fd[i] for i in idx])
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    # colours enter linearly: dI/dc_t is the image of triangle t's weights
    cp = cols.copy()
    cp[3] += 1e-3
    fdc = (np.sum(wts * oracle.shade(m, oracle.setup64(tris), cp, pix)) -
           np.sum(wts * oracle.shade(m, oracle.setup64(tris), cols, pix))) / 1e-3
    assert abs(g["dcolors"][3] - fdc) <= 1e-8 * max(1.0, abs(fdc))


def test_coverage_and_depth_gradients_match_finite_differences():
    tris, cols, W, H, rng = _small_case(seed=11)
    m, eff = oracle.make_map(W, H, 0.4, 0.8, 0.9, 200.0)
    pix = np.arange(W * H)
    dc = rng.normal(size=W * H)
    dd = rng.normal(size=W * H)
    g = oracle.render_grad(m, eff, tris, cols, None, pixels=pix, dcov=dc, ddepth=dd)

    def total(v):
        r = oracle.raster(m, oracle.setup64(v), pix)
        return np.sum(dc * r["cov"]) + np.sum(dd * np.where(np.isfinite(r["depth"]), r["depth"], 0.0))

    h = 1e-6
    a, b = [], []
    for t in range(tris.shape[0]):
        for v in range(3):
            for c in range(3):
                vp, vm = tris.copy(), tris.copy()
                vp[t, v, c] += h
                vm[t, v, c] -= h
                b.append((total(vp) - total(vm)) / (2 * h))
                a.append(g["dtris"][t, v, c])
    a, b = np.array(a), np.array(b)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_homogeneity_identities():
    tris, cols, W, H, rng = _small_case(seed=5, T=20)
    m, eff = oracle.make_map(W, H, 0.3, 0.9, 0.95, 220.0)
    pix = np.arange(W * H)
    g = oracle.render_grad(m, eff, tris, cols, rng.normal(size=W * H), pixels=pix)
    euler = np.sum(g["dtris"] * tris)
    assert abs(euler) <= 1e-12 * np.sum(np.abs(g["dtris"] * tris))
    dd = rng.normal(size=W * H)
    g = oracle.render_grad(m, eff, tris, cols, None, pixels=pix, ddepth=dd)
    r = oracle.raster(m, oracle.setup64(tris), pix)
    depth = np.where(np.isfinite(r["depth"]), r["depth"], 0.0)
    assert np.isclose(np.sum(g["dtris"] * tris), np.sum(dd * depth), rtol=1e-12)


def test_merge_adjoint_on_a_two_triangle_stack():
    # a large near triangle over a larger far one on the optical axis: in the
    # near triangle's ramp the image is m1 s1 + (1 - m1) s2, so moving the near
    # triangle's edge changes the image by (s1 - s2) dm1 -- the FD pin sees
    # the sign of s1 - s2 flip with the colours
    near = np.array([[[-0.2, -0.2, 1.0], [0.3, -0.2, 1.0], [-0.2, 0.3, 1.0]]])
    far = np.array([[[-2.0, -2.0, 3.0], [2.0, -2.0, 3.0], [0.0, 2.0, 3.0]]])
    tris = np.concatenate([near, far])
    W = H = 32
    m, eff = oracle.make_map(W, H, 1.0, 1.0, 1.0, 90.0)
    pix = np.arange(W * H)
    for cols in (np.array([1.0, 0.25]), np.array([0.25, 1.0])):
        g = oracle.render_grad(m, eff, tris, cols, np.ones(W * H), pixels=pix)
        fd = oracle.shade_fd(tris, cols, {"k": 1.0, "l": 1.0, "s": 1.0, "omega": 90.0}, pix, W, H, which=(),
                             vert_idx=[(0, 1, 0)])
        assert np.isclose(g["dtris"][0, 1, 0], fd[(0, 1, 0)], rtol=1e-6)
        # moving the near triangle's right vertex outwards grows it: the image
        # gains where the near colour is the brighter one
        assert np.sign(g["dtris"][0, 1, 0]) == np.sign(cols[0] - cols[1])


@pytest.mark.parametrize("which", ["start", "target"])
def test_grad_workload_crop_against_finite_differences(which):
    # the differentiation workload (1024 x 1024, 10,000 triangles) on a
    # 64 x 64 crop: lens and vertex gradients within 1e-3 relative of FP64
    # central differences
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    lens = start if which == "start" else target
    verts = noisy if which == "start" else tris
    verts = verts.astype(np.float64)
    m, eff = oracle.make_map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
    j0, i0 = 480, 700
    crop = np.array([(j0 + j) * W + i0 + i for j in range(64) for i in range(64)])
    rng = np.random.default_rng(42)
    wts = rng.normal(size=crop.size)
    g = oracle.render_grad(m, eff, verts, colors, wts, pixels=crop)

    def total(ln):
        mm, _ = oracle.make_map(W, H, ln["k"], ln["l"], ln["s"], ln["omega"])
        return float(np.sum(wts * oracle.shade(mm, oracle.setup64(verts), colors, crop)))

    gl = np.array([_fd_lens(lens, n, total) for n in ("k", "l", "s", "omega")])
    scale = np.abs(gl).max()
    assert np.all(np.abs(g["dlens"] - gl) <= 1e-3 * np.abs(gl) + 1e-6 * scale), (g["dlens"], gl)
    touch = np.nonzero(np.abs(g["dtris"]).sum(axis=(1, 2)))[0]
    assert touch.size > 20
    idx = [(t, v, c) for t in touch[:8] for v in range(3) for c in range(3)]
    fd = oracle.shade_fd(verts, colors, lens, crop, W, H, which=(), vert_idx=idx, weights=wts)
    a = np.array([g["dtris"][i] for i in idx])
    b = np.array([fd[i] for i in idx])
    assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_shade_forward_closed_forms():
    # a triangle in the plane z = D facing the eye, pinhole map: inside, away
    # from the ramps, I = c |N-hat . G| = c G_z; behind a fully covering near
    # triangle the far one contributes nothing; and the merge weights add up
    # to the coverage of the order-free merge
    W = H = 32
    m, _ = oracle.make_map(W, H, 1.0, 1.0, 1.0, 90.0)
    near = np.array([[[-3.0, -3.0, 2.0], [3.0, -3.0, 2.0], [0.0, 3.0, 2.0]]])
    far = np.array([[[-9.0, -9.0, 5.0], [9.0, -9.0, 5.0], [0.0, 9.0, 5.0]]])
    G = m.reshape(-1, 4)
    r = oracle.raster(m, oracle.setup64(near))
    full = (r["cov"].ravel() == 1.0)
    img = oracle.shade(m, oracle.setup64(near), np.array([0.7])).ravel()
    assert full.sum() > 100
    assert np.allclose(img[full], 0.7 * G[full, 2], rtol=0, atol=1e-15)
    both = np.concatenate([near, far])
    img2 = oracle.shade(m, oracle.setup64(both), np.array([0.7, 0.3])).ravel()
    assert np.allclose(img2[full], 0.7 * G[full, 2], rtol=0, atol=1e-15)
    # with unit shades (colour 1 / |N-hat . G| is not per pixel, so use the
    # bound instead): 0 <= I <= cov * max c, equality for equal colours on
    # planes facing the eye at the map's centre pixel
    tris, cols, W2, H2, _ = _small_case(seed=3, T=30)
    m2, _ = oracle.make_map(W2, H2, 0.4, 0.8, 0.9, 200.0)
    rec = oracle.setup64(tris)
    img3 = oracle.shade(m2, rec, cols)
    cov = oracle.raster(m2, rec)["cov"]
    assert np.all(img3 >= 0) and np.all(img3 <= cov * cols.max() + 1e-12)
