"""GPU maps of the other projections (Sec. 2.2) and of lens distortion
(Sec. 2.3) against the oracle's, and the raster through them: parity on
sampled pixels against the oracle on the same FP32 map, watertightness of
a closed icosphere, and the differentiable path on such a map."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = [
    ("rectilinear", 1, (100.0,), (), 160, 96),
    ("rectilinear_distorted", 1, (100.0,), (-0.12, 0.03, 0.01, -0.02, 0.005, 0.004), 160, 96),
    ("universal_distorted", 0, (0.32, 0.62, 0.86, 270.0), (-0.05, 0.01, 0.0, 0.0, 0.0, 0.0), 192, 108),
    ("panorama", 2, (300.0, 1.2), (), 192, 80),
    ("dome", 3, (40.0, 20.0, 0.1), (), 128, 128),
    ("equirect", 4, (), (), 256, 128),
    ("cube", 5, (), (), 288, 48),
]


@pytest.fixture(scope="module")
def vsr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10558_gb300 import build, vsr as V
    build.build()
    V.load()
    return V


@pytest.mark.parametrize("name,kind,param,dist,W,H", KINDS)
def test_map_matches_oracle(vsr, name, kind, param, dist, W, H):
    m = vsr.Map.from_spec(kind, W, H, param, dist)
    g = m.download().astype(np.float64)
    if kind == 0:
        eff = oracle.limits(*param)
        o = oracle.make_map_spec(W, H, kind, eff, dist)
    else:
        o = oracle.make_map_spec(W, H, kind, param, dist)
    vg, vo = g[..., 3] > 0, o[..., 3] > 0
    if kind == 3:  # the dome's rim R = 1: FP32 rounding of R may flip a pixel
        fx = 2 * (np.arange(W) + 0.5) / W - 1
        fy = 1 - 2 * (np.arange(H) + 0.5) / H
        R = np.hypot(*np.meshgrid(fx, fy))
        rim = np.abs(R - 1) < 1e-6
        assert np.array_equal(vg[~rim], vo[~rim])
    else:
        assert np.array_equal(vg, vo)
    both = vg & vo
    a, b = g[..., :3][both], o[..., :3][both]
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.einsum("ij,ij->i", a, b))
    assert ang.max() < 2e-6, ang.max()
    assert np.abs(np.linalg.norm(a, axis=-1) - 1).max() < 4e-7
    rel = np.abs(g[..., 3][both] / o[..., 3][both] - 1)
    assert rel.max() < 2e-3, rel.max()


@pytest.mark.parametrize("name,kind,param,dist,W,H", [k for k in KINDS if k[0] in ("cube", "equirect", "dome")])
def test_watertight_icosphere_on_gpu_map(vsr, name, kind, param, dist, W, H):
    m = vsr.Map.from_spec(kind, W, H, param, dist)
    sc = vsr.Scene(torch.from_numpy(scenes.icosphere(4, 50.0)).cuda())
    out = vsr.raster(m, sc, n_inside=True)
    valid = m.download()[..., 3] > 0
    n = out["n_inside"].cpu().numpy()
    assert np.all(n[valid] == 1) and np.all(n[~valid] == 0)
    assert vsr.last_device_status() == 0


@pytest.mark.parametrize("name,kind,param,dist,W,H", [k for k in KINDS if k[0] in ("cube", "panorama",
                                                                                   "rectilinear_distorted")])
def test_raster_through_map_matches_oracle(vsr, name, kind, param, dist, W, H):
    from _util import compare
    m = vsr.Map.from_spec(kind, W, H, param, dist)
    m32 = m.download()
    tris = scenes.random_triangles(3000, 1.0, 20.0, 0.08, seed=21)
    sc = vsr.Scene(torch.from_numpy(tris).cuda())
    out = vsr.raster(m, sc)
    got = {"id": out["id"].cpu().numpy().view(np.uint32), "depth": out["depth"].cpu().numpy(),
           "cov": out["cov"].cpu().numpy()}
    pix = np.random.default_rng(5).integers(0, W * H, 2000)
    rec = oracle.setup(tris)
    exp = oracle.raster(m32, rec, pixels=pix)
    compare(m32, rec, exp, got, pixels=pix)


def test_differentiable_path_on_a_cube_map(vsr):
    W, H = 192, 32
    m = vsr.Map.from_spec(vsr.MAP_CUBE, W, H)
    tris = scenes.random_triangles(500, 1.0, 5.0, 0.2, seed=22)
    colors = np.random.default_rng(1).uniform(0.2, 1.0, 500).astype(np.float32)
    td = torch.from_numpy(tris).cuda()
    cd = torch.from_numpy(colors).cuda()
    sc = vsr.Scene(td)
    fr = vsr.Frags()
    out = vsr.raster_shaded(m, sc, fr, cd)
    img = oracle.shade(m.download().astype(np.float64), oracle.setup(tris), colors.astype(np.float64))
    assert np.abs(out["image"].cpu().numpy() - img).max() <= 1e-5
    # vertex gradients exist, the lens gradient does not (no lens parameters)
    g = vsr.raster_backward(m, sc, fr, td, cd, out["id"], dimage=torch.ones((H, W), device="cuda"),
                            want=("tris",))
    assert torch.isfinite(g["dtris"]).all() and g["dtris"].abs().max() > 0
    with pytest.raises(vsr.VsrError):
        vsr.raster_backward(m, sc, fr, td, cd, out["id"], dimage=torch.ones((H, W), device="cuda"), want=("lens",))


def test_invalid_specs_are_refused(vsr):
    for kind, param in [(6, ()), (-1, ()), (1, (180.0,)), (1, (0.0,)), (2, (0.0, 1.0)), (0, (float("nan"), 1, 1, 90))]:
        with pytest.raises(vsr.VsrError):
            vsr.Map.from_spec(kind, 64, 64, param)
    with pytest.raises(vsr.VsrError):
        vsr.Map.from_spec(vsr.MAP_CUBE, 0, 64)
    with pytest.raises(vsr.VsrError):
        vsr.Map.from_spec(vsr.MAP_UNIVERSAL, 64, 64, (0.0, 1.0, 1.0, 180.0), distortion=(float("inf"),))
    # an empty scene through a generated map and through pstep
    m = vsr.Map.from_spec(vsr.MAP_EQUIRECT, 64, 32, derivatives=True)
    sc = vsr.Scene(torch.zeros((0, 3, 3), dtype=torch.float32, device="cuda"))
    for out in (vsr.raster(m, sc), vsr.raster_pstep(m, sc)):
        assert (out["id"].cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all()
        assert float(out["cov"].abs().max()) == 0.0
    assert vsr.last_device_status() == 0
