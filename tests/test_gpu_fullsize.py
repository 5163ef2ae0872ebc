"""Full-size parity of the batched and served paths against the FP64 oracle.

Views of the batched workload itself -- 2048 x 1024 and 1920 x 1080 maps,
k < 0 lenses whose rim pixels are invalid (asin out of its domain), angles
of view of 304 and 320 deg, an eye 0.9 from the origin inside the cloud --
rendered by vsr_batch_render over the workload's 1,000,000-triangle scene.
Per view, 4096 seeded pixels and one seeded 128 x 128 crop are computed one
by one by the oracle on the same FP32 map (the oracle's FP64 map rounded
once, an input of the rasterizer) and compared under the parity rules.  One
request of the serving workload's distribution goes through vsr_serve_* on
its own GPU-made map and is held to the same rules."""
import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

from _util import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VIEWS = [0, 3, 12, 15, 43, 60]  # indices into scenes.batched_views()


@pytest.fixture(scope="module")
def vsr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10558_gb300 import build, vsr as V
    build.build()
    V.load()
    return V


@pytest.fixture(scope="module")
def scene():
    return scenes.batched_scene()


def _sample(W, H, seed):
    """4096 seeded pixels plus one seeded 128 x 128 crop (flat indices)."""
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, W * H, 4096)
    x0, y0 = int(rng.integers(0, W - 128)), int(rng.integers(0, H - 128))
    yy, xx = np.meshgrid(np.arange(y0, y0 + 128), np.arange(x0, x0 + 128), indexing="ij")
    return np.unique(np.concatenate([pix, (yy * W + xx).ravel()]))


def _np(o):
    return {"id": o["id"].cpu().numpy().view(np.uint32), "depth": o["depth"].cpu().numpy(),
            "cov": o["cov"].cpu().numpy()}


def test_batched_full_size_against_oracle(vsr, scene):
    views = [scenes.batched_views()[i] for i in VIEWS]
    tris = torch.from_numpy(scene).cuda()
    m32s, maps = [], []
    for v in views:
        m64, _ = oracle.make_map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"])
        m32s.append(m64.astype(np.float32))
        maps.append(vsr.Map.from_tensor(torch.from_numpy(m32s[-1]).cuda()))
    outs = [{"id": torch.empty((v["H"], v["W"]), dtype=torch.int32, device="cuda"),
             "depth": torch.empty((v["H"], v["W"]), dtype=torch.float32, device="cuda"),
             "cov": torch.empty((v["H"], v["W"]), dtype=torch.float32, device="cuda")} for v in views]
    b = vsr.Batch()
    b.render(maps, tris, np.stack([v["cam"] for v in views]), outs)
    assert vsr.last_device_status() == 0
    worst = {"cov_max_err": 0.0, "depth_max_rel": 0.0, "id_equal_frac": 1.0}
    n_invalid = 0
    for i, v, m32, o in zip(VIEWS, views, m32s, outs):
        pix = _sample(v["W"], v["H"], seed=100 + i)
        rec = oracle.setup(scene, v["cam"])
        exp = oracle.raster(m32, rec, pixels=pix)
        rep = compare(m32, rec, exp, _np(o), pixels=pix)
        n_invalid += len(pix) - rep["n_valid"]
        print(f"batched view {i} ({v['W']}x{v['H']}, k={v['k']:.2f}, Omega={v['omega']:.0f}): {rep}")
        worst["cov_max_err"] = max(worst["cov_max_err"], rep["cov_max_err"])
        worst["depth_max_rel"] = max(worst["depth_max_rel"], rep["depth_max_rel"])
        worst["id_equal_frac"] = min(worst["id_equal_frac"], rep["id_equal_frac"])
    print(f"batched full size, worst over {len(VIEWS)} views: {worst}")
    assert n_invalid > 0  # the k < 0 rims were sampled


def test_served_full_size_against_oracle(vsr, scene):
    """View 43 of the batched workload (1920 x 1080, k = -0.51, Omega = 320
    deg, invalid rim) served from the 1M-triangle scene next to other
    requests; the server makes its own map, which equals a vsr_make_map map
    of the same lens bit for bit, so the oracle reads that map."""
    v = scenes.batched_views()[43]
    tris = torch.from_numpy(scene).cuda()
    srv = vsr.Server(budget_bytes=8 << 30, slots=4)
    try:
        sid = srv.add_scene(tris)
        small = torch.from_numpy(scenes.random_triangles(20000, 1.0, 30.0, 0.03, seed=8)).cuda()
        sid2 = srv.add_scene(small)
        npx = v["W"] * v["H"]
        out = {k: torch.empty(npx, dtype=dt, device="cuda")
               for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32))}
        others = [{k: torch.empty(512 * 512, dtype=dt, device="cuda")
                   for k, dt in (("id", torch.int32), ("depth", torch.float32), ("cov", torch.float32))}
                  for _ in range(3)]
        lens = dict(W=v["W"], H=v["H"], k=v["k"], l=v["l"], s=v["s"], omega=v["omega"])
        tickets = [srv.submit(sid2, dict(W=512, H=512, k=0.3, l=0.8, s=0.9, omega=200.0), scenes.camera(), o)
                   for o in others[:2]]
        t = srv.submit(sid, lens, v["cam"], out)
        tickets.append(srv.submit(sid2, dict(W=512, H=512, k=-0.2, l=0.9, s=0.7, omega=250.0), scenes.camera(),
                                  others[2]))
        r = srv.wait(t)
        for q in tickets:
            assert srv.wait(q)["status"] == 0
        assert r["status"] == 0
    finally:
        srv.close()
    got = {k: out[k].view(v["H"], v["W"]) for k in out}
    m = vsr.Map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"])
    m32 = m.download()
    ref = _np(vsr.raster(m, vsr.Scene(tris, v["cam"])))
    got_np = _np(got)
    for k in ("id", "depth", "cov"):  # the served result is the plain path's on that map
        assert np.array_equal(got_np[k].view(np.uint32), ref[k].view(np.uint32)), k
    pix = _sample(v["W"], v["H"], seed=243)
    rec = oracle.setup(scene, v["cam"])
    exp = oracle.raster(m32, rec, pixels=pix)
    rep = compare(m32, rec, exp, got_np, pixels=pix)
    print(f"served view 43 ({v['W']}x{v['H']}): {rep}")
    assert rep["n_valid"] < len(pix)
