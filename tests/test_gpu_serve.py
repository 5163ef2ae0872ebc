"""The rendering server (vsr_serve_*): continuous batching over several
streams, the map cache, the memory budget, cancellation -- and each result
equal to the same request rendered alone."""
import numpy as np
import pytest

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


def _out(lens):
    return {"id": torch.empty((lens["H"], lens["W"]), dtype=torch.int32, device="cuda"),
            "depth": torch.empty((lens["H"], lens["W"]), dtype=torch.float32, device="cuda"),
            "cov": torch.empty((lens["H"], lens["W"]), dtype=torch.float32, device="cuda")}


def _lens_pool(n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(128, 96), (160, 160), (200, 100), (97, 61)]
    return [dict(W=sizes[i % 4][0], H=sizes[i % 4][1], k=float(rng.uniform(-1, 1)), l=float(rng.uniform(0.5, 1)),
                 s=float(rng.uniform(0.5, 1)), omega=float(rng.uniform(90, 360))) for i in range(n)]


def test_results_alone_equal_results_in_the_mix(vsr):
    sc_np = [scenes.random_triangles(3000, 1.0, 20.0, 0.05, seed=30),
             scenes.random_triangles(12000, 1.0, 40.0, 0.02, seed=31)]
    sc = [torch.from_numpy(t).cuda() for t in sc_np]
    srv = vsr.Server(budget_bytes=8 << 30, slots=4)
    ids = [srv.add_scene(t) for t in sc]
    pool = _lens_pool(6, seed=3)
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(48):
        lens = pool[int(rng.integers(len(pool)))]
        cam = scenes.camera(rng.uniform(-1, 1, 3))
        s = int(rng.integers(2))
        out = _out(lens)
        reqs.append((s, lens, cam, out, srv.submit(ids[s], lens, cam, out)))
    for s, lens, cam, out, t in reqs:
        r = srv.wait(t)
        assert r["done"] and r["status"] == 0 and r["t_done"] >= r["t_start"] >= r["t_submit"]
    st = srv.stats()
    assert st["completed"] == 48 and st["map_hits"] > 0 and st["map_misses"] <= len(pool)
    torch.cuda.synchronize()
    for s, lens, cam, out, t in reqs:
        m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
        alone = vsr.raster(m, vsr.Scene(sc[s], cam))
        for k in ("id", "depth", "cov"):
            assert torch.equal(alone[k], out[k]), k
    srv.close()


def test_growing_map_shape_reruns_without_blocking(vsr):
    """One slot, so one workspace per scene: a small map, then maps with
    many times its tile count.  The workspace keeps its bins' capacity
    across shapes instead of waiting for the device to size them, so the
    larger maps outgrow it; the server renders those requests again with
    grown bins, and every result equals the plain path's."""
    tris = torch.from_numpy(scenes.random_triangles(12000, 1.0, 40.0, 0.02, seed=31)).cuda()
    srv = vsr.Server(budget_bytes=8 << 30, slots=1)
    sid = srv.add_scene(tris)
    lenses = [dict(W=64, H=48, k=0.2, l=0.9, s=0.9, omega=120.0),
              dict(W=1024, H=1024, k=-0.3, l=0.8, s=0.7, omega=300.0),
              dict(W=2048, H=1024, k=0.5, l=0.7, s=0.9, omega=250.0),
              dict(W=64, H=48, k=0.2, l=0.9, s=0.9, omega=120.0)]
    outs, tickets = [], []
    for lens in lenses:
        out = _out(lens)
        outs.append(out)
        tickets.append(srv.submit(sid, lens, scenes.camera(), out))
    for t in tickets:
        assert srv.wait(t)["status"] == 0
    st = srv.stats()
    srv.close()
    assert st["reruns"] >= 1, st
    torch.cuda.synchronize()
    for lens, out in zip(lenses, outs):
        m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
        alone = vsr.raster(m, vsr.Scene(tris, scenes.camera()))
        for k in ("id", "depth", "cov"):
            assert torch.equal(alone[k], out[k]), (lens["W"], k)


def test_cached_map_shared_while_it_is_made(vsr):
    """Requests on other slots that take a map from the cache while the slot
    that made it is still generating it (a 2048 x 2048 map, scenes of a few
    hundred triangles whose set-up ends long before the map) must wait for
    it: every result equals the same request rendered alone."""
    tris = torch.from_numpy(scenes.random_triangles(400, 1.0, 20.0, 0.05, seed=7)).cuda()
    lens = dict(W=2048, H=2048, k=0.3, l=0.8, s=0.9, omega=200.0)
    srv = vsr.Server(budget_bytes=8 << 30, slots=4)
    sid = srv.add_scene(tris)
    rng = np.random.default_rng(8)
    reqs = []
    for _ in range(8):
        cam = scenes.camera(rng.uniform(-0.5, 0.5, 3))
        out = _out(lens)
        reqs.append((cam, out, srv.submit(sid, lens, cam, out)))
    for cam, out, t in reqs:
        r = srv.wait(t)
        assert r["done"] and r["status"] == 0
    st = srv.stats()
    assert st["map_misses"] == 1 and st["map_hits"] == 7
    torch.cuda.synchronize()
    m = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    for cam, out, t in reqs:
        alone = vsr.raster(m, vsr.Scene(tris, cam))
        for k in ("id", "depth", "cov"):
            assert torch.equal(alone[k], out[k]), k
    srv.close()


def test_budget_cancel_and_invalid(vsr):
    tris = torch.from_numpy(scenes.random_triangles(2000, 1.0, 20.0, 0.05, seed=5)).cuda()
    lens = dict(W=256, H=256, k=0.0, l=1.0, s=1.0, omega=180.0)
    # a budget below one map: rejected at submission
    tiny = vsr.Server(budget_bytes=1 << 20, slots=1)
    s0 = tiny.add_scene(tris)
    with pytest.raises(vsr.VsrError) as e:
        tiny.submit(s0, lens, scenes.camera(), _out(lens))
    assert e.value.code == -7
    tiny.close()
    # room for the map but not for the workspace: fails when admitted
    small = vsr.Server(budget_bytes=1_300_000 + 256 * 256 * 16, slots=1)
    s1 = small.add_scene(tris)
    r = small.wait(small.submit(s1, lens, scenes.camera(), _out(lens)))
    assert r["done"] and r["status"] == -7
    small.close()
    # cancellation of queued requests; invalid parameters
    srv = vsr.Server(budget_bytes=4 << 30, slots=1)
    s2 = srv.add_scene(tris)
    outs = [_out(lens) for _ in range(30)]
    tickets = [srv.submit(s2, lens, scenes.camera([0.01 * i, 0, 0]), o) for i, o in enumerate(outs)]
    cancelled = [t for t in tickets[10:] if srv.cancel(t)]
    assert cancelled
    for t in tickets:
        r = srv.wait(t)
        assert r["status"] in (0, -8) and (r["status"] == -8) == (t in cancelled)
    bad = dict(lens, k=float("nan"))
    with pytest.raises(vsr.VsrError):
        srv.submit(s2, bad, scenes.camera(), outs[0])
    with pytest.raises(vsr.VsrError):
        srv.submit(99, lens, scenes.camera(), outs[0])
    assert srv.stats()["cancelled"] == len(cancelled)
    srv.close()
