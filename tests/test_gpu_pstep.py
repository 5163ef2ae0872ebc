"""GPU rasterization with the per-fragment pixel step (vsr_raster_pstep)
against the oracle's pstep raster on the GPU's own FP32 map and
differences, under the parity rules of the coverage kernel; watertightness
and complementary ramps of a closed mesh under pstep."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

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


def _np(o):
    return {"id": o["id"].cpu().numpy().view(np.uint32), "depth": o["depth"].cpu().numpy(),
            "cov": o["cov"].cpu().numpy()}


@pytest.mark.parametrize("case", ["tiny", "universal", "cube", "small_tris"])
def test_pstep_matches_oracle(vsr, case):
    from _util import compare
    if case == "tiny":
        lens, tris, _cam = scenes.tiny_scene()
        m = vsr.Map.from_spec(vsr.MAP_UNIVERSAL, lens["W"], lens["H"],
                              (lens["k"], lens["l"], lens["s"], lens["omega"]), derivatives=True)
        pix = None
    elif case == "universal":
        m = vsr.Map.from_spec(vsr.MAP_UNIVERSAL, 320, 180, (0.32, 0.62, 0.86, 270.0), derivatives=True)
        tris = scenes.random_triangles(20000, 1.0, 40.0, 0.05, seed=41)
        pix = np.random.default_rng(1).integers(0, 320 * 180, 3000)
    elif case == "cube":
        m = vsr.Map.from_spec(vsr.MAP_CUBE, 288, 48, derivatives=True)
        tris = scenes.random_triangles(5000, 1.0, 20.0, 0.08, seed=42)
        pix = np.random.default_rng(2).integers(0, 288 * 48, 3000)
    else:  # caps far below a pixel: the wide pstep miter region
        m = vsr.Map.from_spec(vsr.MAP_UNIVERSAL, 128, 96, (0.0, 1.0, 1.0, 120.0), derivatives=True)
        tris = scenes.random_triangles(3000, 1.0, 10.0, 0.002, seed=43)
        pix = None
    sc = vsr.Scene(torch.from_numpy(tris).cuda())
    got = _np(vsr.raster_pstep(m, sc))
    assert vsr.last_device_status() == 0
    m32 = m.download()
    d32 = m.download_derivatives()
    rec = oracle.setup(tris)
    exp = oracle.raster_pstep(m32, d32, rec, pixels=pix)
    compare(m32, rec, exp, got, pixels=pix)


def test_pstep_closed_mesh(vsr):
    W, H = 320, 180
    m = vsr.Map.from_spec(vsr.MAP_UNIVERSAL, W, H, (0.32, 0.62, 0.86, 270.0), derivatives=True)
    tris = scenes.icosphere(4, 50.0)
    sc = vsr.Scene(torch.from_numpy(tris).cuda())
    ref = vsr.raster(m, sc)  # global step, its own bins
    out = vsr.raster_pstep(m, sc)
    cov = out["cov"].cpu().numpy()
    g = m.download()
    valid = g[..., 3] > 0
    V = np.unique(tris.reshape(-1, 3).astype(np.float64), axis=0)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    G = g[..., :3].reshape(-1, 3).astype(np.float64)
    near = np.zeros(W * H, dtype=bool)
    for a in range(0, V.shape[0], 512):  # within 3 ramp widths of a vertex
        near |= (np.arccos(np.clip(G @ V[a:a + 512].T, -1, 1)) * g[..., 3].reshape(-1, 1) < 3.0).any(1)
    ok = valid.ravel() & ~near
    assert np.abs(cov.ravel()[ok] - 1).max() < 2e-6
    # the global-step raster may reuse the (wider) pstep bins: same outputs
    again = vsr.raster(m, sc, binned=True)
    for k in ("id", "depth", "cov"):
        assert np.array_equal(ref[k].cpu().numpy(), again[k].cpu().numpy()), k
    assert vsr.last_device_status() == 0


def test_pstep_needs_derivatives(vsr):
    m = vsr.Map(64, 64, 0.0, 1.0, 1.0, 180.0)
    sc = vsr.Scene(torch.from_numpy(scenes.random_triangles(10, 1.0, 5.0, 0.1, seed=1)).cuda())
    with pytest.raises(vsr.VsrError):
        vsr.raster_pstep(m, sc)
