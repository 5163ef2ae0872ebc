"""CUDA path versus the FP64 oracle, through the C ABI (libvsr.so).

Raster parity feeds both sides the same map: the oracle's FP64 map rounded
to FP32 once, uploaded with vsr_map_from_device (the map is an input of the
rasterizer).  Map parity compares the GPU's own map with the oracle's.
The end-to-end check (GPU map + GPU raster against oracle map + oracle
raster) carries the map's rounding into coverage and is held to the looser
bound derived from it."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

from _util import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vsr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10558_gb300 import build, vsr as V
    build.build()
    V.load()
    return V


def _gpu_outputs(out):
    return {"id": out["id"].cpu().numpy().view(np.uint32), "depth": out["depth"].cpu().numpy(),
            "cov": out["cov"].cpu().numpy()}


def _oracle_map32(lens, aov=0):
    m64, eff = oracle.make_map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"], aov=aov)
    return m64.astype(np.float32), eff


def _raster_shared_map(V, lens, tris, cam, pixels=None, stats=False):
    m32, _ = _oracle_map32(lens)
    gm = V.Map.from_tensor(torch.from_numpy(m32).cuda())
    sc = V.Scene(torch.from_numpy(tris).cuda(), cam)
    out = V.raster(gm, sc, stats=stats)
    assert V.last_device_status() == 0
    rec = oracle.setup(tris, cam)
    exp = oracle.raster(m32, rec, pixels=pixels)
    return m32, rec, exp, out


# ---------------------------------------------------------------------------
# map

MAP_CASES = [
    dict(W=256, H=256, k=0.0, l=1.0, s=1.0, omega=180.0),
    dict(W=1920, H=1080, k=0.32, l=0.62, s=0.86, omega=270.0),
    dict(W=333, H=197, k=-1.0, l=1.0, s=1.0, omega=180.0),
    dict(W=512, H=512, k=-0.5, l=0.8, s=0.6, omega=360.0),
    dict(W=640, H=480, k=1.0, l=1.0, s=1.0, omega=120.0),
    dict(W=300, H=200, k=0.0, l=0.5, s=0.7, omega=360.0),
]

# FP32 map function: tan/atan/asin/sin/cos each within a few ulp, so the
# direction is off by at most ~8 ulp of theta (<= pi): 8 * 2^-24 * pi ~ 1.5e-6.
MAP_ANGLE_TOL = 2e-6
# delta is a central difference of neighbouring FP32 directions ~1/delta
# apart: relative error ~ (2 x 1.5e-6 rad) x delta, bounded below at 1e-3 for
# the resolutions tested.
MAP_DELTA_TOL = 2e-3


def _asin_condition(lens, eff):
    """For k < 0, theta = asin(sin(k Omega/2) R)/k amplifies the FP32 rounding
    of its argument by 1/sqrt(1 - arg^2) near the rim; 1 elsewhere."""
    W, H = lens["W"], lens["H"]
    i, j = np.meshgrid(np.arange(W), np.arange(H))
    x = 2 * (i + 0.5) / W - 1
    y = (2 * (j + 0.5) / H - 1) * H / W
    R = np.sqrt(x * x + eff[1] * y * y)
    if eff[0] >= 0:
        return np.ones_like(R)
    arg = np.abs(np.sin(eff[0] * math.radians(eff[3]) / 2) * R)
    return np.maximum(1.0, 0.25 / np.sqrt(np.maximum(1e-12, 1 - np.minimum(arg, 1) ** 2)))


def _angle(a, b):
    """Angle between direction fields, insensitive to their lengths."""
    c = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(c, (a * b).sum(-1))


@pytest.mark.parametrize("lens", MAP_CASES, ids=lambda d: f"{d['W']}x{d['H']}k{d['k']}")
def test_map_parity(vsr, lens):
    gm = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    got = gm.download().astype(np.float64)
    exp, eff = oracle.make_map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    p = gm.params()
    assert abs(p["omega_deg"] - eff[3]) < 1e-4 and abs(p["k"] - eff[0]) < 1e-7
    ve, vg = exp[..., 3] > 0, got[..., 3] > 0
    both = ve & vg
    # validity differs only on the asin domain edge (|sin(k Omega/2) R| ~ 1)
    assert (ve != vg).sum() <= max(2, 1e-4 * ve.size)
    ang = _angle(exp[..., :3], got[..., :3])
    tol = MAP_ANGLE_TOL * _asin_condition(lens, eff)
    assert (ang - tol)[both].max() < 0, (ang / tol)[both].max()
    assert np.abs(np.linalg.norm(got[..., :3], axis=-1) - 1)[vg].max() < 4e-7
    rel = np.abs(got[..., 3] / np.where(both, exp[..., 3], 1.0) - 1.0)
    assert rel[both].max() < MAP_DELTA_TOL, rel[both].max()
    assert np.all(got[~vg] == 0.0)


def test_map_aov_types(vsr):
    for aov in (1, 2, 3):
        lens = dict(W=200, H=120, k=0.32, l=0.62, s=0.86, omega=200.0)
        gm = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"], aov=aov)
        got = gm.download().astype(np.float64)
        exp, _ = oracle.make_map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"], aov=aov)
        both = (exp[..., 3] > 0) & (got[..., 3] > 0)
        assert _angle(exp[..., :3], got[..., :3])[both].max() < MAP_ANGLE_TOL


# ---------------------------------------------------------------------------
# raster, shared FP32 map

def test_raster_parity_tiny(vsr):
    """256x256 equidistant view of 64 seeded triangles, full frame."""
    lens, tris, cam = scenes.tiny_scene()
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, cam, stats=True)
    rep = compare(m32, rec, exp, _gpu_outputs(out))
    assert out["n_alg"] == exp["n_alg"] or abs(out["n_alg"] - exp["n_alg"]) <= 1e-5 * exp["n_alg"]
    assert rep["n_valid"] == 256 * 256


@pytest.mark.parametrize("lens", [dict(W=333, H=197, k=-1.0, l=1.0, s=1.0, omega=180.0),
                                  dict(W=300, H=200, k=0.0, l=0.5, s=0.7, omega=360.0),
                                  dict(W=97, H=61, k=1.0, l=1.0, s=1.0, omega=150.0),
                                  dict(W=1, H=1, k=0.0, l=1.0, s=1.0, omega=90.0),
                                  dict(W=17, H=300, k=0.6, l=0.9, s=0.9, omega=250.0)],
                         ids=["ortho-invalid-corners", "wrap360", "ragged-pinhole", "1x1", "tall"])
def test_raster_parity_lenses(vsr, lens):
    """Ragged tiles, invalid pixels, wrap-around beyond 180 deg, degenerate
    sizes; scenes with small, large and near-eye triangles."""
    tris = np.concatenate([scenes.random_triangles(150, 1.0, 10.0, 0.25, seed=5),
                           scenes.random_triangles(150, 2.0, 30.0, 0.03, seed=6),
                           scenes.random_triangles(5, 0.05, 0.2, 1.2, seed=7)])
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, scenes.camera())
    compare(m32, rec, exp, _gpu_outputs(out))


def test_raster_parity_camera_and_culling(vsr):
    """Moved and rotated camera; culled triangles (vertex at the eye,
    collinear with the eye) are never drawn."""
    lens = dict(W=320, H=240, k=0.5, l=0.8, s=0.9, omega=220.0)
    tris = scenes.random_triangles(400, 1.0, 10.0, 0.2, seed=12)
    O = np.array([0.3, -0.2, 0.5], dtype=np.float32)
    th = 0.4
    M = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    cam = scenes.camera(O, M)
    bad = np.array([[O, O + [1, 0, 0], O + [0, 1, 0]], [O + [1, 0, 1], O + [2, 0, 2], O + [0, 1, 3]]],
                   dtype=np.float32)
    tris = np.concatenate([tris, bad])
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, cam)
    compare(m32, rec, exp, _gpu_outputs(out))
    ids = out["id"].cpu().numpy().view(np.uint32)
    assert not np.isin(ids, [len(tris) - 2, len(tris) - 1]).any()


def test_raster_empty_scene(vsr):
    m = vsr.Map(64, 48, 0.0, 1.0, 1.0, 180.0)
    sc = vsr.Scene(torch.zeros((0, 3, 3), dtype=torch.float32, device="cuda"))
    out = vsr.raster(m, sc)
    assert (out["id"].cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all()
    assert torch.isinf(out["depth"]).all() and (out["cov"] == 0).all()


def test_single_view_workload_sampled(vsr):
    """The 1920x1080 single-view workload (icosphere + 200k triangles) in the
    launch configuration the benchmark times; the oracle checks 4096 seeded
    pixels and a 96x96 crop one by one."""
    lens, tris, cam = scenes.single_view_scene()
    rng = np.random.default_rng(99)
    W, H = lens["W"], lens["H"]
    pix = rng.integers(0, W * H, 4096)
    cj, ci = 500, 900
    crop = (np.arange(cj, cj + 96)[:, None] * W + np.arange(ci, ci + 96)[None, :]).ravel()
    pixels = np.concatenate([pix, crop])
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, cam, pixels=pixels)
    rep = compare(m32, rec, exp, _gpu_outputs(out), pixels=pixels)
    assert rep["n_valid"] == len(pixels)


def test_regenerated_map_equals_fresh_map(vsr):
    """A map regenerated in place (vsr_map_update, same size) through lenses
    of very different tile sizes, each twice: the binner's widest ramp comes
    from the map kernels' generation-tagged maximum, never from an earlier
    generation, so every frame equals that of a freshly made map of the same
    lens, bit for bit."""
    W, H = 640, 360
    lenses = [(0.32, 0.62, 0.86, 270.0), (-0.5, 0.8, 0.6, 200.0), (1.0, 1.0, 1.0, 100.0), (0.0, 0.5, 0.7, 360.0),
              (0.32, 0.62, 0.86, 270.0)]
    tris = scenes.random_triangles(3000, 1.0, 20.0, 0.03, seed=23)
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(W, H, *lenses[0])
    for lens in lenses:
        fresh = _gpu_outputs(vsr.raster(vsr.Map(W, H, *lens), sc))
        for _ in range(2):
            m.update(W, H, *lens)
            got = _gpu_outputs(vsr.raster(m, sc))
            assert vsr.last_device_status() == 0
            for k in got:
                assert np.array_equal(got[k].view(np.uint32), fresh[k].view(np.uint32)), (lens, k)


@pytest.mark.parametrize("lens", [dict(W=256, H=256, k=0.0, l=1.0, s=1.0, omega=180.0),
                                  dict(W=333, H=197, k=-1.0, l=1.0, s=1.0, omega=180.0),
                                  dict(W=300, H=200, k=0.0, l=0.5, s=0.7, omega=360.0),
                                  dict(W=320, H=240, k=1.0, l=1.0, s=1.0, omega=60.0)],
                         ids=lambda d: f"{d['W']}x{d['H']}k{d['k']}o{d['omega']:.0f}")
def test_dense_reference_equals_binned(vsr, lens):
    """vsr_raster_dense (every pixel against every triangle, no tile bins)
    gives vsr_raster's outputs bit for bit: ragged tiles, invalid corners, a
    360-degree wrap, a 60-degree view that most triangles miss (the binner
    skips caps outside the map's field of view), triangles culled at set-up
    (a vertex at the eye, a plane through it) and more than one chunk of
    triangles per tile."""
    tris = np.concatenate([scenes.random_triangles(900, 1.0, 10.0, 0.15, seed=31),
                           scenes.random_triangles(300, 0.5, 3.0, 0.4, seed=32)])
    tris[5, 0] = 0.0                       # a vertex at the eye
    tris[6, 2] = 2.0 * tris[6, 0]          # A, B, C on one line through the eye... 
    tris[6, 1] = 3.0 * tris[6, 0]          # ...so the plane holds the eye (det = 0)
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    binned = _gpu_outputs(vsr.raster(m, sc))
    dense = _gpu_outputs(vsr.raster_dense(m, sc))
    assert vsr.last_device_status() == 0
    for k in binned:
        assert np.array_equal(binned[k].view(np.uint32), dense[k].view(np.uint32)), k
    assert (binned["id"] != oracle.NO_ID).mean() > 0.2


@pytest.mark.parametrize("jitter", [0.1, 0.7], ids=["coarse_grid", "large_list"])
def test_heavy_tiles_equal_dense(vsr, jitter):
    """2500 triangles near the eye with wide caps -- past the fine grid's two
    cells (coarse grid) or past the coarse grid's (the list every tile
    tests: every tile's window then holds more candidates than one warp
    stages, and each tile is binned by a whole CTA) -- among 3000 ordinary
    ones, few per tile, so the scene is binned tile-major.  The binned
    outputs equal the dense reference's bit for bit."""
    near = scenes.random_triangles(2500, 0.05, 0.3, jitter, seed=42)
    tris = np.concatenate([scenes.random_triangles(3000, 1.0, 20.0, 0.02, seed=41), near])
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(256, 256, 0.32, 0.62, 0.86, 300.0)
    binned = _gpu_outputs(vsr.raster(m, sc))
    dense = _gpu_outputs(vsr.raster_dense(m, sc))
    assert vsr.last_device_status() == 0
    for k in binned:
        assert np.array_equal(binned[k].view(np.uint32), dense[k].view(np.uint32)), k
    assert (binned["id"] != oracle.NO_ID).mean() > 0.3


@pytest.mark.parametrize("n", [40000, 200000], ids=["tile_major", "triangle_major"])
def test_binner_choice_equals_dense(vsr, n):
    """The same small wide view over few and over many triangles per tile
    (the scene path bins the first tile-major, the second triangle-major):
    both equal the dense reference bit for bit."""
    tris = scenes.random_triangles(n, 1.0, 20.0, 0.02, seed=43)
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(512, 384, 0.0, 1.0, 1.0, 360.0)
    binned = _gpu_outputs(vsr.raster(m, sc))
    dense = _gpu_outputs(vsr.raster_dense(m, sc))
    assert vsr.last_device_status() == 0
    for k in binned:
        assert np.array_equal(binned[k].view(np.uint32), dense[k].view(np.uint32)), k


def test_large_map_regenerated_equals_fresh_map(vsr):
    """A 4096 x 2176 map (34,816 tiles) updated twice with each of two
    lenses: every frame equals a freshly made map's bit for bit."""
    W, H = 4096, 2176
    lens_a, lens_b = (0.0, 1.0, 1.0, 180.0), (0.32, 0.62, 0.86, 270.0)
    tris = scenes.random_triangles(4000, 1.0, 20.0, 0.05, seed=24)
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(W, H, *lens_a)
    for lens in (lens_a, lens_b):
        fresh = _gpu_outputs(vsr.raster(vsr.Map(W, H, *lens), sc))
        for _ in range(2):
            m.update(W, H, *lens)
            got = _gpu_outputs(vsr.raster(m, sc))
            assert vsr.last_device_status() == 0
            for k in got:
                assert np.array_equal(got[k].view(np.uint32), fresh[k].view(np.uint32)), (lens, k)


def test_large_map_against_oracle(vsr):
    """A 4096 x 2176 map (34,816 tiles, 9.1 Mpx): sampled pixels against the
    oracle."""
    lens = dict(W=4096, H=2176, k=0.0, l=1.0, s=1.0, omega=180.0)
    tris = scenes.random_triangles(2000, 1.0, 20.0, 0.05, seed=21)
    rng = np.random.default_rng(22)
    pixels = rng.integers(0, lens["W"] * lens["H"], 4096)
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, scenes.camera(), pixels=pixels)
    rep = compare(m32, rec, exp, _gpu_outputs(out), pixels=pixels)
    assert rep["n_valid"] == len(pixels)


def test_watertight_icosphere_gpu_map(vsr):
    """Level-5 icosphere around the eye on the GPU's own 1080p map: exactly
    one centre-inside triangle per pixel, coverage 1 away from vertices."""
    W, H = 1920, 1080
    tris = scenes.icosphere(5, 50.0)
    m = vsr.Map(W, H, 0.32, 0.62, 0.86, 270.0)
    sc = vsr.Scene(torch.from_numpy(tris).cuda())
    out = vsr.raster(m, sc, n_inside=True)
    n_in = out["n_inside"].cpu().numpy()
    mp = m.download().astype(np.float64)
    valid = mp[..., 3] > 0
    assert (n_in[valid] == 1).all(), np.unique(n_in[valid], return_counts=True)
    cov = out["cov"].cpu().numpy()
    verts = np.unique(tris.reshape(-1, 3), axis=0).astype(np.float64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    # distance to the nearest vertex direction, in pixels, on a sample
    rng = np.random.default_rng(3)
    pick = rng.integers(0, W * H, 20000)
    G = mp.reshape(-1, 4)[pick, :3]
    d = np.arccos(np.clip((G @ verts.T).max(1), -1, 1)) * mp.reshape(-1, 4)[pick, 3]
    far = d > 2.5
    assert far.mean() > 0.3
    assert np.abs(cov.reshape(-1)[pick][far] - 1).max() < 1e-5


def test_end_to_end_against_oracle(vsr):
    """GPU map + GPU raster against oracle map + oracle raster.  The map's
    FP32 rounding (<= 2e-6 rad) moves edge distances by as much, i.e. coverage
    by delta x 2e-6 (delta ~ 80 here), and delta's own rounding scales ramps by
    <= 2e-3: coverage is held to 2e-3 and ids to 99.9 %."""
    lens, tris, cam = scenes.tiny_scene()
    m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), cam)
    got = _gpu_outputs(vsr.raster(m, sc))
    m64, _ = oracle.make_map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    exp = oracle.raster(m64, oracle.setup(tris, cam))
    assert np.abs(got["cov"] - exp["cov"]).max() < 2e-3
    assert (got["id"] == exp["id"]).mean() > 0.999


def test_bins_resized_for_a_new_map_shape(vsr):
    """One scene rendered twice on a small map -- the second binning leaves
    its pair total unread -- then on a map with 340 times the tiles: the
    bins are sized from the new frame's own total, and the frame equals a
    fresh scene's with no overflow reported."""
    tris = torch.from_numpy(scenes.random_triangles(20000, 1.0, 30.0, 0.03, seed=25)).cuda()
    sc = vsr.Scene(tris, scenes.camera())
    small = vsr.Map(64, 48, 0.2, 0.9, 0.9, 120.0)
    big = vsr.Map(1920, 1080, 0.32, 0.62, 0.86, 270.0)
    for _ in range(2):
        vsr.raster(small, sc)
    got = _gpu_outputs(vsr.raster(big, sc))
    assert vsr.last_device_status() == 0
    ref = _gpu_outputs(vsr.raster(big, vsr.Scene(tris, scenes.camera())))
    for k in got:
        assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), k


def test_deterministic(vsr):
    lens, tris, cam = scenes.tiny_scene()
    m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), cam)
    a = _gpu_outputs(vsr.raster(m, sc))
    b = _gpu_outputs(vsr.raster(m, sc))
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32))


def test_render_host_matches_device_path(vsr):
    lens, tris, cam = scenes.tiny_scene()
    m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    dev = _gpu_outputs(vsr.raster(m, vsr.Scene(torch.from_numpy(tris).cuda(), cam)))
    work = vsr.Scene()
    for _ in range(2):
        host = vsr.render_host(m, work, tris, cam)
        for k in dev:
            assert np.array_equal(dev[k].view(np.uint32), host[k].view(np.uint32))


def test_render_host_pinned_in_place(vsr):
    """Pinned (mapped) host buffers are read and written in place by the
    kernels; the outputs equal the device path's bit for bit, also when only
    some buffers are pinned (the rest staged)."""
    lens, tris, cam = scenes.tiny_scene()
    H, W = lens["H"], lens["W"]
    m = vsr.Map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
    dev = _gpu_outputs(vsr.raster(m, vsr.Scene(torch.from_numpy(tris).cuda(), cam)))
    tris_pin = torch.from_numpy(tris).pin_memory().numpy()
    work = vsr.Scene()
    for pin_outputs in (("id", "depth", "cov"), ("cov",), ()):
        out = {}
        for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32)):
            buf = torch.full((H, W), 7, dtype=dt)
            out[k] = (buf.pin_memory() if k in pin_outputs else buf).numpy()
        out["id"] = out["id"].view(np.uint32)
        for _ in range(2):
            host = vsr.render_host(m, work, tris_pin, cam, out=out)
            for k in dev:
                assert np.array_equal(dev[k].view(np.uint32), host[k].view(np.uint32)), (pin_outputs, k)
    # pageable triangles with pinned outputs
    out = {k: torch.zeros((H, W), dtype=dt).pin_memory().numpy()
           for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32))}
    out["id"] = out["id"].view(np.uint32)
    host = vsr.render_host(m, work, tris, cam, out=out)
    for k in dev:
        assert np.array_equal(dev[k].view(np.uint32), host[k].view(np.uint32))


def test_render_host_beside_map_update(vsr):
    """A lens's map update is queued on the stream just before
    vsr_render_host, whose set-up runs beside it on the scene's own stream;
    once, a use of the work scene queued on another stream in between must be
    waited for.  Every frame equals vsr_raster on a fresh map of the same lens
    bit for bit (ragged 333 x 197 tiles, outputs written in place in whole
    tile rows, split tiles)."""
    W, H = 333, 197
    tris = scenes.random_triangles(30000, 1.0, 30.0, 0.03, seed=21)
    cam = scenes.camera()
    td = torch.from_numpy(tris).cuda()
    lenses = [(0.3, 0.8, 0.9, 200.0), (-0.4, 0.7, 0.8, 250.0), (0.0, 1.0, 1.0, 120.0)]
    tris_pin = torch.from_numpy(tris).pin_memory().numpy()
    out = {k: torch.zeros((H, W), dtype=dt).pin_memory().numpy()
           for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32))}
    out["id"] = out["id"].view(np.uint32)
    m = vsr.Map(W, H, *lenses[0])
    work = vsr.Scene()
    side = torch.cuda.Stream()
    for i, lens in enumerate(lenses * 2):
        m.update(W, H, *lens)
        if i == 3:
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                kept = vsr.raster(m, work, stream=side)  # noqa: F841 (outputs live past the call)
        host = vsr.render_host(m, work, tris_pin, cam, out=out)
        ref = _gpu_outputs(vsr.raster(vsr.Map(W, H, *lens), vsr.Scene(td, cam)))
        for k in ref:
            assert np.array_equal(ref[k].view(np.uint32), host[k].view(np.uint32)), (i, k)
    assert vsr.last_device_status() == 0


def test_render_host_async_pipeline(vsr):
    """Frames queued with vsr_render_host_async on two (map, scene) pairs in
    turn, each pair on its own stream, overlap on the device; each frame,
    once waited for, equals vsr_raster on a fresh map of its lens bit for bit.
    A frame that outgrew its scene's bins is reported by the wait
    (VSR_ERR_BIN_OVERFLOW) and rendered again; a second queue on a scene whose
    frame was not waited for is refused."""
    W, H = 333, 197
    tris = scenes.random_triangles(30000, 1.0, 30.0, 0.03, seed=21)
    cam = scenes.camera()
    td = torch.from_numpy(tris).cuda()
    lenses = [(0.3, 0.8, 0.9, 200.0), (-0.4, 0.7, 0.8, 250.0), (0.0, 1.0, 1.0, 120.0), (0.6, 0.9, 0.7, 300.0)] * 2
    tris_pin = torch.from_numpy(tris).pin_memory().numpy()

    def pinned_outputs():
        o = {k: torch.zeros((H, W), dtype=dt).pin_memory().numpy()
             for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32))}
        o["id"] = o["id"].view(np.uint32)
        return o

    outs = [pinned_outputs(), pinned_outputs()]
    maps = [vsr.Map(W, H, *lenses[0]), vsr.Map(W, H, *lenses[1])]
    works = [vsr.Scene(), vsr.Scene()]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pending = [None, None]
    overflowed = []

    def finish(i):
        k, lens = pending[i]
        pending[i] = None
        if vsr.render_host_wait(works[i]) == vsr.VSR_ERR_BIN_OVERFLOW:
            overflowed.append(k)
            vsr.render_host(maps[i], works[i], tris_pin, cam, out=outs[i], stream=streams[i])
        ref = _gpu_outputs(vsr.raster(vsr.Map(W, H, *lens), vsr.Scene(td, cam)))
        for key in ref:
            assert np.array_equal(ref[key].view(np.uint32), outs[i][key].view(np.uint32)), (k, key)

    for k, lens in enumerate(lenses):
        i = k % 2
        if pending[i] is not None:
            finish(i)
        maps[i].update(W, H, *lens, stream=streams[i])
        vsr.render_host_async(maps[i], works[i], tris_pin, cam, out=outs[i], stream=streams[i])
        pending[i] = (k, lens)
        if k == 2:
            with pytest.raises(vsr.VsrError):
                vsr.render_host_async(maps[i], works[i], tris_pin, cam, out=outs[i], stream=streams[i])
    for i in (0, 1):
        if pending[i] is not None:
            finish(i)
    assert vsr.render_host_wait(works[0]) == 0  # nothing queued
    assert vsr.last_device_status() == 0
    print("frames rendered again after a bin overflow:", overflowed)


def test_invalid_arguments(vsr):
    L = vsr.load()
    import ctypes
    h = ctypes.c_void_p()
    assert L.vsr_make_map(float("nan"), 1, 1, 90, 64, 64, None, ctypes.byref(h)) == -1
    assert L.vsr_make_map(0.0, 1, 1, 90, 0, 64, None, ctypes.byref(h)) == -1
    assert L.vsr_make_map(0.0, 1, 1, 90, 64, 40000, None, ctypes.byref(h)) == -1
    assert L.vsr_raster(None, None, None, None, None, None) == -1
    cam = (ctypes.c_float * 12)(*([float("inf")] + [0.0] * 11))
    assert L.vsr_setup(None, 0, cam, None, ctypes.byref(h)) == -1
    assert L.vsr_last_device_status() == 0


def test_split_tiles_against_oracle_and_unsplit(vsr):
    """Thousands of triangles stacked over a few tiles: bins far longer than
    one work item, so the tiles are split over several CTAs whose results
    merge with atomics.  Checked against the oracle (sampled pixels) and bit
    for bit against the unsplit diagnostic kernel."""
    rng = np.random.default_rng(17)
    n = 3000
    c = np.stack([rng.normal(0, 0.05, n), rng.normal(0, 0.05, n), np.ones(n)], 1)
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    rho = rng.uniform(2.0, 20.0, n)
    t1 = np.cross(c, [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(c, t1)
    uv = rng.uniform(-0.06, 0.06, (n, 3, 2))
    d = c[:, None, :] + uv[..., 0:1] * t1[:, None, :] + uv[..., 1:2] * t2[:, None, :]
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    tris = (rho[:, None, None] * d).astype(np.float32)
    lens = dict(W=96, H=80, k=0.0, l=1.0, s=1.0, omega=40.0)
    m32, rec, exp, out = _raster_shared_map(vsr, lens, tris, scenes.camera(), pixels=np.arange(0, 96 * 80, 7))
    got = _gpu_outputs(out)
    compare(m32, rec, exp, got, pixels=np.arange(0, 96 * 80, 7))
    # the same map and scene through the unsplit per-tile kernel (statistics path)
    gm = vsr.Map.from_tensor(torch.from_numpy(m32).cuda())
    sc = vsr.Scene(torch.from_numpy(tris).cuda())
    vsr.bin(gm, sc)
    # 3000 triangles inside ~0.15 rad of the axis over 16-px tiles of ~0.12 rad:
    # the central bins hold well over one work item (512) each
    assert sc.bin_pairs() > 3 * n
    a = _gpu_outputs(vsr.raster(gm, sc, binned=True))
    b = _gpu_outputs(vsr.raster(gm, sc, binned=True, stats="exec"))
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k

