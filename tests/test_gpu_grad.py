"""GPU parity of the differentiable path (vsr_raster_shaded /
vsr_raster_backward) against the FP64 oracle.

Forward: the shaded image (front-to-back merge of c_t |N-hat . G|), the
merge coverage, id and depth, against oracle.shade / oracle.raster on the
GPU's own FP32 map and the same FP32 vertices, and against vsr_raster.
Backward: vertex, colour and lens gradients against the oracle's analytic
FP64 adjoint on the same FP32 inputs, and against FP64 central differences
of the oracle (h = 1e-6, vertices in float64) on a 64 x 64 crop of the
1024 x 1024 differentiation workload, within 1e-3 relative."""

import numpy as np
import pytest

import oracle
from paper_2003_10558_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5     # absolute, image values are <= max colour <= 1
COV_TOL = 1e-5
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def vsr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10558_gb300 import build, vsr as V
    build.build()
    V.load()
    return V


def _crop(W, j0, i0, n=64):
    return np.array([(j0 + j) * W + i0 + i for j in range(n) for i in range(n)], dtype=np.int64)


def _forward(V, lens, tris, colors):
    W, H = lens["W"], lens["H"]
    r = V.ShadedRenderer(W, H)
    eff = r.set_lens(lens["k"], lens["l"], lens["s"], lens["omega"])
    tris_d = torch.from_numpy(np.ascontiguousarray(tris)).cuda()
    col_d = torch.from_numpy(np.ascontiguousarray(colors)).cuda()
    r.scene.update(tris_d, r.cam)
    out = V.raster_shaded(r.map, r.scene, r.frags, col_d)
    torch.cuda.synchronize()
    return r, eff, tris_d, col_d, out


def _check_forward(V, r, out, tris, colors, pix=None):
    m64 = r.map.download().astype(np.float64)
    rec = oracle.setup(tris)
    img = out["image"].cpu().numpy().ravel()
    cov = out["cov"].cpu().numpy().ravel()
    o_img = oracle.shade(m64, rec, colors.astype(np.float64), pix)
    o = oracle.raster(m64, rec, pix)
    sel = slice(None) if pix is None else pix
    d_img = np.abs(img[sel] - o_img.ravel())
    d_cov = np.abs(cov[sel] - o["cov"].ravel())
    assert d_img.max() <= IMG_TOL, (d_img.max(), np.argmax(d_img))
    assert d_cov.max() <= COV_TOL, d_cov.max()
    # id and depth as the coverage kernel's
    ref = V.raster(r.map, r.scene)
    assert np.array_equal(out["id"].cpu().numpy(), ref["id"].cpu().numpy())
    assert np.array_equal(out["depth"].cpu().numpy(), ref["depth"].cpu().numpy())
    assert np.abs(out["cov"].cpu().numpy() - ref["cov"].cpu().numpy()).max() <= 2e-6
    assert V.last_device_status() == 0


def test_shaded_forward_tiny_full_frame(vsr):
    lens, tris, _cam = scenes.tiny_scene()
    colors = np.random.default_rng(0).uniform(0.2, 1.0, tris.shape[0]).astype(np.float32)
    r, _eff, _t, _c, out = _forward(vsr, lens, tris, colors)
    _check_forward(vsr, r, out, tris, colors)


def test_shaded_forward_grad_workload_sampled(vsr):
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    r, _eff, _t, _c, out = _forward(vsr, start, noisy, colors)
    rng = np.random.default_rng(4)
    pix = np.unique(np.concatenate([_crop(W, 480, 700), _crop(W, 0, 0, 32), rng.integers(0, W * H, 4096)]))
    _check_forward(vsr, r, out, noisy, colors, pix)


def _gpu_grads(V, r, tris_d, col_d, out, dimage=None, dcov=None, ddepth=None):
    g = V.raster_backward(r.map, r.scene, r.frags, tris_d, col_d, out["id"], dimage, dcov, ddepth)
    torch.cuda.synchronize()
    assert V.last_device_status() == 0
    return {k: v.cpu().numpy() for k, v in g.items()}


def _upstream(W, H, crop, seed):
    rng = np.random.default_rng(seed)
    w = np.zeros(W * H, dtype=np.float32)
    w[crop] = rng.normal(size=crop.size).astype(np.float32)
    return w


def _close(a, b, rtol=GRAD_RTOL):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) <= rtol * np.linalg.norm(b) + 1e-12


@pytest.mark.parametrize("which", ["start", "target"])
def test_backward_matches_oracle_gradient(vsr, which):
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    lens = start if which == "start" else target
    verts = noisy if which == "start" else tris
    r, eff, tris_d, col_d, out = _forward(vsr, lens, verts, colors)
    crop = _crop(W, 480, 700)
    w = _upstream(W, H, crop, 11)
    g = _gpu_grads(vsr, r, tris_d, col_d, out, dimage=torch.from_numpy(w).cuda().view(H, W))
    m64 = r.map.download().astype(np.float64)
    o = oracle.render_grad(m64, eff, verts.astype(np.float64), colors.astype(np.float64), w[crop].astype(np.float64),
                           pixels=crop)
    touch = np.nonzero(np.abs(o["dtris"]).sum(axis=(1, 2)))[0]
    assert touch.size > 20
    assert _close(g["dtris"][touch], o["dtris"][touch])
    # no gradient where the oracle has none
    rest = np.setdiff1d(np.arange(verts.shape[0]), touch)
    assert np.abs(g["dtris"][rest]).max() <= 1e-6 * np.abs(o["dtris"]).max()
    assert _close(g["dcolors"], o["dcolors"])
    for j in range(4):
        assert abs(g["dlens"][j] - o["dlens"][j]) <= GRAD_RTOL * abs(o["dlens"][j]) + 1e-6 * np.abs(o["dlens"]).max(), \
            (j, g["dlens"], o["dlens"])


def test_coverage_and_depth_adjoints_match_oracle(vsr):
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    r, eff, tris_d, col_d, out = _forward(vsr, target, tris, colors)
    crop = _crop(W, 300, 300)
    dc = _upstream(W, H, crop, 12)
    dd = _upstream(W, H, crop, 13)
    g = _gpu_grads(vsr, r, tris_d, col_d, out, dcov=torch.from_numpy(dc).cuda().view(H, W),
                   ddepth=torch.from_numpy(dd).cuda().view(H, W))
    m64 = r.map.download().astype(np.float64)
    o = oracle.render_grad(m64, eff, tris.astype(np.float64), colors.astype(np.float64), None, pixels=crop,
                           dcov=dc[crop].astype(np.float64), ddepth=dd[crop].astype(np.float64))
    assert _close(g["dtris"], o["dtris"])
    for j in range(4):
        assert abs(g["dlens"][j] - o["dlens"][j]) <= GRAD_RTOL * abs(o["dlens"][j]) + 1e-6 * np.abs(o["dlens"]).max()


def test_backward_against_fp64_finite_differences(vsr):
    # the differentiation workload's bar: GPU gradient (FP32 forward, FP32
    # adjoint) against FP64 central differences of the oracle, h = 1e-6, on a
    # 64 x 64 crop, relative error < 1e-3
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    r, eff, tris_d, col_d, out = _forward(vsr, start, noisy, colors)
    crop = _crop(W, 480, 700)
    w = _upstream(W, H, crop, 11)
    g = _gpu_grads(vsr, r, tris_d, col_d, out, dimage=torch.from_numpy(w).cuda().view(H, W))
    verts = noisy.astype(np.float64)
    wc = w[crop].astype(np.float64)

    def total(ln):
        mm, _ = oracle.make_map(W, H, ln["k"], ln["l"], ln["s"], ln["omega"])
        return float(np.sum(wc * oracle.shade(mm, oracle.setup64(verts), colors.astype(np.float64), crop)))

    h = 1e-6
    fd = {}
    for name in ("k", "l", "s", "omega"):
        lp, lm = dict(start), dict(start)
        if name in ("l", "s") and start[name] + h > 1.0:  # at the upper limit: one-sided from inside
            lm2 = dict(start)
            lm[name] -= h
            lm2[name] -= 2 * h
            fd[name] = (3 * total(start) - 4 * total(lm) + total(lm2)) / (2 * h)
        else:
            lp[name] += h
            lm[name] -= h
            fd[name] = (total(lp) - total(lm)) / (2 * h)
    gl = np.array([fd[n] for n in ("k", "l", "s", "omega")])
    scale = np.abs(gl).max()
    for j in range(4):
        assert abs(g["dlens"][j] - gl[j]) <= GRAD_RTOL * abs(gl[j]) + 1e-6 * scale, (j, g["dlens"], gl)
    touch = np.nonzero(np.abs(g["dtris"]).sum(axis=(1, 2)))[0][:8]
    idx = [(t, v, c) for t in touch for v in range(3) for c in range(3)]
    fdv = oracle.shade_fd(verts, colors.astype(np.float64), start, crop, W, H, which=(), vert_idx=idx, weights=wc)
    a = np.array([g["dtris"][i] for i in idx])
    b = np.array([fdv[i] for i in idx])
    assert _close(a, b)


def test_autograd_function_and_stale_backward(vsr):
    target, start, tris, noisy, colors, W, H = scenes.grad_scene(W=256, H=256)
    r = vsr.ShadedRenderer(W, H)
    tris_d = torch.from_numpy(noisy).cuda().requires_grad_(True)
    col_d = torch.from_numpy(colors).cuda().requires_grad_(True)
    lens = torch.tensor([start["k"], start["l"], start["s"], start["omega"]], dtype=torch.float64,
                        requires_grad=True)
    tgt = torch.rand((H, W), device="cuda")
    img, cov, depth, ids = vsr.render_shaded(tris_d, col_d, lens, r)
    loss = ((img - tgt) ** 2).sum()
    loss.backward()
    assert lens.grad is not None and lens.grad.dtype == torch.float64 and torch.isfinite(lens.grad).all()
    # l = s = 1 are at the limits but unclamped: their gradients are kept
    # (l's is the one-sided derivative from inside); the same gradients
    # through the raw ABI
    g = vsr.raster_backward(r.map, r.scene, r.frags, tris_d.detach(), col_d.detach(), ids,
                            dimage=2 * (img.detach() - tgt))
    # (per-triangle sums are float atomics: two runs agree to their rounding)
    def same(a, b):
        return torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))

    assert same(tris_d.grad, g["dtris"])
    assert same(col_d.grad, g["dcolors"])
    assert same(lens.grad, g["dlens"].cpu())
    # a clamped parameter gets no gradient
    lens2 = torch.tensor([start["k"], 1.5, start["s"], start["omega"]], dtype=torch.float64, requires_grad=True)
    img2, *_ = vsr.render_shaded(tris_d, col_d, lens2, r)
    img2.sum().backward()
    assert lens2.grad[1].item() == 0.0 and lens2.grad[0].item() != 0.0
    # backward of an older forward of the same renderer is refused
    img3, *_ = vsr.render_shaded(tris_d, col_d, lens, r)
    img4, *_ = vsr.render_shaded(tris_d, col_d, lens, r)
    with pytest.raises(vsr.VsrError):
        img3.sum().backward()
    img4.sum().backward()


def test_lens_fit_recovers_target(vsr):
    # the differentiation workload at 256 x 256: start (0.6, 1, 1) with
    # vertex noise, target rendered at (0.2, 0.7, 0.9) from the true vertices
    from paper_2003_10558_gb300 import fit
    target, start, tris, noisy, colors, W, H = scenes.grad_scene(W=256, H=256)
    r = vsr.ShadedRenderer(W, H)
    col = torch.from_numpy(colors).cuda()
    lt = torch.tensor([target["k"], target["l"], target["s"], target["omega"]], dtype=torch.float64)
    with torch.no_grad():
        tgt = vsr.render_shaded(torch.from_numpy(tris).cuda(), col, lt, r)[0].clone()
    res = fit.fit_lens(tgt, torch.from_numpy(noisy).cuda(), col, start, r, steps=30, vertex_steps=30)
    got = res["lens"]
    assert abs(got["k"] - 0.2) < 0.01 and abs(got["l"] - 0.7) < 0.01 and abs(got["s"] - 0.9) < 0.01, got
    first_full = next(h[1] for h in res["history"] if h[0] == 0)
    assert res["history"][-1][1] < first_full  # the vertex stage lowers the full-resolution loss


def test_lens_fit_full_size_workload(vsr):
    """The differentiation workload at its own size: 1024 x 1024, 10,000
    triangles, start (0.6, 1, 1) with N(0, 0.01^2) vertex noise, target
    rendered at (0.2, 0.7, 0.9) from the true vertices.  The coarse-to-fine
    fit recovers the lens within 0.01."""
    from paper_2003_10558_gb300 import fit
    target, start, tris, noisy, colors, W, H = scenes.grad_scene()
    assert (W, H, len(tris)) == (1024, 1024, 10_000)
    r = vsr.ShadedRenderer(W, H)
    col = torch.from_numpy(colors).cuda()
    lt = torch.tensor([target["k"], target["l"], target["s"], target["omega"]], dtype=torch.float64)
    with torch.no_grad():
        tgt = vsr.render_shaded(torch.from_numpy(tris).cuda(), col, lt, r)[0].clone()
    res = fit.fit_lens(tgt, torch.from_numpy(noisy).cuda(), col, start, r, steps=30, vertex_steps=30)
    got = res["lens"]
    print(f"fit 1024^2: {got} in {len(res['history'])} steps, {res['seconds']:.2f} s")
    assert abs(got["k"] - 0.2) < 0.01 and abs(got["l"] - 0.7) < 0.01 and abs(got["s"] - 0.9) < 0.01, got


def test_lens_fit_checkpoint_resume(vsr, tmp_path):
    """A fit saved after any step and loaded into a fresh LensFit continues
    where it stopped.  The lens stages are deterministic: a resumed run
    repeats the uninterrupted one bit for bit (loss, k, l, s of every step,
    the final lens and Adam moments).  The vertex stage sums per-triangle
    gradients with float atomics: its state is restored bit for bit, and the
    continued steps agree with the uninterrupted run to rounding."""
    from paper_2003_10558_gb300 import fit
    target, start, tris, noisy, colors, W, H = scenes.grad_scene(W=256, H=256)
    col = torch.from_numpy(colors).cuda()
    lt = torch.tensor([target["k"], target["l"], target["s"], target["omega"]], dtype=torch.float64)
    r = vsr.ShadedRenderer(W, H)
    with torch.no_grad():
        tgt = vsr.render_shaded(torch.from_numpy(tris).cuda(), col, lt, r)[0].clone()
    nz = torch.from_numpy(noisy).cuda()
    kw = dict(sigmas=(16, 4, 0), steps=8, vertex_steps=6)

    def make():
        return fit.LensFit(tgt, nz, col, start, vsr.ShadedRenderer(W, H), **kw)

    full = make().run()
    again = make().run(max_steps=24)  # the lens stages of a second uninterrupted run
    assert full.history[:24] == again.history  # deterministic lens stages
    # stop inside the second lens stage, save, resume in a fresh fit
    a = make().run(max_steps=11)
    path = tmp_path / "fit.pt"
    a.save(path)
    b = make().load(path)
    sa, sb = a.state_dict(), b.state_dict()
    assert torch.equal(sa["lens"], sb["lens"]) and torch.equal(sa["verts"], sb["verts"])
    assert (b.stage, b.step_in_stage) == (1, 3)
    b.run(max_steps=13)  # to the end of the lens stages
    assert b.history == full.history[:24]
    ma = full.opt.state_dict()["state"][0]
    mb = b.opt.state_dict()["state"][0]
    assert torch.equal(ma["exp_avg"], mb["exp_avg"]) and torch.equal(ma["exp_avg_sq"], mb["exp_avg_sq"])
    # into the vertex stage: save after two of its steps, resume
    b.run(max_steps=2)
    b.save(path)
    c = make().load(path)
    assert torch.equal(c.verts.detach(), b.verts.detach()) and c.stage == 3 and c.step_in_stage == 2
    c.run()
    assert c.done() and len(c.history) == len(full.history)
    for hc, hf in zip(c.history, full.history):
        assert abs(hc[1] - hf[1]) <= 1e-4 * abs(hf[1]) and max(abs(x - y) for x, y in zip(hc[2:], hf[2:])) < 1e-5
    with pytest.raises(ValueError):
        fit.LensFit(tgt, nz, col, start, r, sigmas=(8, 0), steps=8, vertex_steps=6).load(path)


def test_empty_scene_and_invalid_calls(vsr):
    W, H = 64, 48
    r = vsr.ShadedRenderer(W, H)
    r.set_lens(0.3, 0.8, 0.9, 200.0)
    empty = torch.zeros((0, 3, 3), dtype=torch.float32, device="cuda")
    cols = torch.zeros((0,), dtype=torch.float32, device="cuda")
    r.scene.update(empty, r.cam)
    out = vsr.raster_shaded(r.map, r.scene, r.frags, cols)
    assert float(out["image"].abs().max()) == 0.0 and float(out["cov"].abs().max()) == 0.0
    assert (out["id"].cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all()
    g = vsr.raster_backward(r.map, r.scene, r.frags, empty, cols, out["id"],
                            dimage=torch.ones((H, W), device="cuda"))
    assert g["dtris"].numel() == 0 and float(g["dlens"].abs().max()) == 0.0
    assert vsr.last_device_status() == 0
    # a backward for a map or scene changed since the forward is refused
    r.set_lens(0.2, 0.8, 0.9, 200.0)
    with pytest.raises(vsr.VsrError):
        vsr.raster_backward(r.map, r.scene, r.frags, empty, cols, out["id"], dimage=torch.ones((H, W), device="cuda"))
