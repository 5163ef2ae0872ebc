"""Batched multi-view rendering (one CUDA graph of per-view chains over
parallel streams) against per-view vsr_raster calls and the oracle."""
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


def _views(n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(96, 64), (160, 160), (200, 100), (33, 47), (128, 96), (64, 64)]
    out = []
    for v in range(n):
        W, H = sizes[v % len(sizes)]
        out.append(dict(W=W, H=H, k=float(rng.uniform(-1, 1)), l=float(rng.uniform(0.5, 1)),
                        s=float(rng.uniform(0.5, 1)), omega=float(rng.uniform(90, 360)),
                        cam=scenes.camera(rng.uniform(-1.5, 1.5, 3))))
    return out


def _outs(views, dev="cuda"):
    return [{"id": torch.empty((v["H"], v["W"]), dtype=torch.int32, device=dev),
             "depth": torch.empty((v["H"], v["W"]), dtype=torch.float32, device=dev),
             "cov": torch.empty((v["H"], v["W"]), dtype=torch.float32, device=dev)} for v in views]


def _np(o):
    return {k: o[k].cpu().numpy().view(np.uint32) if k == "id" else o[k].cpu().numpy() for k in ("id", "depth", "cov")}


@pytest.mark.parametrize("mode", ["auto", "chains", "pooled"])
def test_batch_equals_per_view_raster(vsr, mode):
    """Each graph kind the autotuner may keep -- per-view raster launches, or
    one pooled persistent launch over all views' work items -- equals
    per-view vsr_raster bit for bit, also after the cameras move."""
    views = _views(6, seed=3)
    tris_np = scenes.random_triangles(20000, 1.0, 30.0, 0.03, seed=8)
    tris = torch.from_numpy(tris_np).cuda()
    maps = [vsr.Map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"]) for v in views]
    b = vsr.Batch()
    b.set_mode({"auto": vsr.Batch.AUTO, "chains": vsr.Batch.CHAINS, "pooled": vsr.Batch.POOLED}[mode])
    outs = _outs(views)
    rng = np.random.default_rng(5)
    for call in range(4):
        if call == 3:  # move every camera: the graph replays with new cameras
            for v in views:
                v["cam"] = scenes.camera(rng.uniform(-1.5, 1.5, 3))
        cams = np.stack([v["cam"] for v in views])
        for o in outs:
            o["id"].fill_(7)
            o["cov"].fill_(-1)
        b.render(maps, tris, cams, outs)
        assert vsr.last_device_status() == 0
        for v, m, o in zip(views, maps, outs):
            ref = _np(vsr.raster(m, vsr.Scene(tris, v["cam"])))
            got = _np(o)
            for k in ("id", "depth", "cov"):
                assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), (call, k)
        if call >= 1:
            assert b.config()["graphed"]
    assert b.config()["streams"] in (1, 2, 4, 6)
    assert b.config()["split_max"] in (256, 512, 1024)
    if mode != "auto":
        assert b.config()["pooled"] == (mode == "pooled")


def test_batch_view_against_oracle(vsr):
    """Sampled pixels of one batched view, computed one by one by the oracle
    on the same (oracle-made, FP32-rounded) map."""
    from _util import compare
    views = _views(3, seed=11)
    tris_np = scenes.random_triangles(5000, 1.0, 20.0, 0.05, seed=12)
    maps, m32s = [], []
    for v in views:
        m64, _ = oracle.make_map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"])
        m32 = m64.astype(np.float32)
        m32s.append(m32)
        maps.append(vsr.Map.from_tensor(torch.from_numpy(m32).cuda()))
    b = vsr.Batch()
    outs = _outs(views)
    b.render(maps, torch.from_numpy(tris_np).cuda(), np.stack([v["cam"] for v in views]), outs)
    assert vsr.last_device_status() == 0
    rng = np.random.default_rng(1)
    for v, m32, o in zip(views, m32s, outs):
        pix = rng.integers(0, v["W"] * v["H"], 600)
        rec = oracle.setup(tris_np, v["cam"])
        exp = oracle.raster(m32, rec, pixels=pix)
        compare(m32, rec, exp, _np(o), pixels=pix)


def test_batch_grows_bins_when_cameras_move(vsr):
    # pinhole views that first look away from the scene (empty bins), then
    # from inside it: the first frame with the new cameras may outgrow the
    # bins (reported in the device status), the next call re-sizes them and
    # renders exactly what per-view vsr_raster renders
    views = [dict(W=128, H=96, k=1.0, l=1.0, s=1.0, omega=90.0) for _ in range(3)]
    tris = torch.from_numpy(scenes.random_triangles(20000, 1.0, 30.0, 0.03, seed=8)).cuda()
    maps = [vsr.Map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"]) for v in views]
    b = vsr.Batch()
    outs = _outs(views)
    far = np.stack([scenes.camera((0.0, 0.0, 200.0 + i)) for i in range(3)])
    near = np.stack([scenes.camera((0.2 * i, 0.0, 0.0)) for i in range(3)])
    b.render(maps, tris, far, outs)
    b.render(maps, tris, far, outs)
    assert vsr.last_device_status() == 0
    b.render(maps, tris, near, outs)
    assert vsr.last_device_status() in (0, vsr.VSR_ERR_BIN_OVERFLOW)
    b.render(maps, tris, near, outs)
    assert vsr.last_device_status() == 0
    for cam, m, o in zip(near, maps, outs):
        ref = _np(vsr.raster(m, vsr.Scene(tris, cam)))
        got = _np(o)
        for k in ("id", "depth", "cov"):
            assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), k
