"""vsr_raster_noalloc: rasterization for callers that cannot allocate device
memory while they render (frameworks that own all device memory, real-time
loops that must not wait on cudaMalloc).  Its bins live in a fixed array
inside the library; the test checks, through the C ABI, that two calls in a
row give the same outputs as vsr_raster within the parity tolerances, that
they allocate nothing, report a clean status, and reject oversized inputs.

This file is collected last on purpose: a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2003_10558_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COV_TOL = 1e-5
DEPTH_TOL = 1e-5


@pytest.fixture(scope="module")
def vsr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10558_gb300 import build, vsr as V
    build.build()
    V.load()
    return V


def _outputs(H, W):
    return (torch.empty((H, W), dtype=torch.int32, device="cuda"),
            torch.empty((H, W), dtype=torch.float32, device="cuda"),
            torch.empty((H, W), dtype=torch.float32, device="cuda"))


def _noalloc(V, m, sc, outs, status):
    L = V.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.vsr_raster_noalloc(m.h, sc.h, ctypes.c_void_p(outs[0].data_ptr()), ctypes.c_void_p(outs[1].data_ptr()),
                              ctypes.c_void_p(outs[2].data_ptr()), ctypes.c_void_p(status.data_ptr()), stream)
    return rc


@pytest.mark.parametrize("workload", ["tiny", "single_view"])
def test_noalloc_matches_raster_twice(vsr, workload):
    if workload == "tiny":
        lens, tris, cam = scenes.tiny_scene()
    else:
        lens, tris, cam = scenes.single_view_scene()
    W, H = lens["W"], lens["H"]
    m = vsr.Map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), cam)
    ref = vsr.raster(m, sc)
    assert vsr.last_device_status() == 0
    ref_id = ref["id"].cpu().numpy().view(np.uint32)
    ref_depth = ref["depth"].cpu().numpy()
    ref_cov = ref["cov"].cpu().numpy()

    outs = _outputs(H, W)
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        outs[0].fill_(7)
        outs[2].fill_(-1.0)
        assert _noalloc(vsr, m, sc, outs, status) == 0
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert int(status.item()) == 0
        gid = outs[0].cpu().numpy().view(np.uint32)
        assert np.array_equal(gid, ref_id)
        assert np.abs(outs[2].cpu().numpy() - ref_cov).max() <= COV_TOL
        hit = ref_id != 0xFFFFFFFF
        d = outs[1].cpu().numpy()
        assert np.abs(d[hit] / ref_depth[hit] - 1).max() <= DEPTH_TOL
        assert np.isinf(d[~hit]).all()


def test_noalloc_after_map_updates(vsr):
    """The fixed-array path builds the map's tile index on its first use
    after each generation of the map: through updates of one map with
    different lenses (and the same lens twice), it matches vsr_raster's
    outputs every time."""
    W, H = 640, 360
    lenses = [(0.32, 0.62, 0.86, 270.0), (-0.5, 0.8, 0.6, 200.0), (-0.5, 0.8, 0.6, 200.0), (1.0, 1.0, 1.0, 100.0)]
    tris = scenes.random_triangles(3000, 1.0, 20.0, 0.03, seed=23)
    sc = vsr.Scene(torch.from_numpy(tris).cuda(), scenes.camera())
    m = vsr.Map(W, H, *lenses[0])
    outs = _outputs(H, W)
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for lens in lenses:
        m.update(W, H, *lens)
        ref = vsr.raster(m, sc)
        assert vsr.last_device_status() == 0
        for _ in range(2):
            assert _noalloc(vsr, m, sc, outs, status) == 0
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            ref_id = ref["id"].cpu().numpy().view(np.uint32)
            assert np.array_equal(outs[0].cpu().numpy().view(np.uint32), ref_id), lens
            assert np.abs(outs[2].cpu().numpy() - ref["cov"].cpu().numpy()).max() <= COV_TOL
            hit = ref_id != 0xFFFFFFFF
            d = outs[1].cpu().numpy()
            assert np.abs(d[hit] / ref["depth"].cpu().numpy()[hit] - 1).max() <= DEPTH_TOL


def test_noalloc_limits(vsr):
    # more tiles than the array holds: refused on the host
    big_map = vsr.Map(4096, 2048, 0.0, 1.0, 1.0, 180.0)
    small = vsr.Scene(torch.from_numpy(scenes.random_triangles(10, 1.0, 10.0, 0.1, seed=4)).cuda())
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    outs = _outputs(2048, 4096)
    assert _noalloc(vsr, big_map, small, outs, status) == -1
    # more (tile, triangle) pairs than the array holds: known only on the
    # device, reported in the status word, no access outside the array
    m = vsr.Map(64, 64, 0.0, 1.0, 1.0, 180.0)
    many = vsr.Scene(torch.from_numpy(scenes.random_triangles(600000, 1.0, 10.0, 0.3, seed=3)).cuda())
    outs = _outputs(64, 64)
    status.fill_(0)
    assert _noalloc(vsr, m, many, outs, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == vsr.VSR_ERR_BIN_OVERFLOW
    # the array is usable again right after
    lens, tris, _cam = scenes.tiny_scene()
    tm = vsr.Map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    ts = vsr.Scene(torch.from_numpy(tris).cuda())
    ref = vsr.raster(tm, ts)
    outs = _outputs(lens["H"], lens["W"])
    assert _noalloc(vsr, tm, ts, outs, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(outs[0].cpu().numpy(), ref["id"].cpu().numpy())
