"""Lens fitting through the differentiable renderer.

Finds the Universal-perspective lens (k, l, s) -- and optionally refines
the triangle vertices -- whose shaded render matches a target image, by
gradient descent on the L2 image loss with the gradients of
vsr_raster_backward (the hand-written adjoint of the shaded image through
the merge, the plane distances, the set-up and the map).

A lens change moves image content by many pixels, farther than the scale
of the scene's detail, so the raw L2 loss is flat far from the answer.  The
fit therefore runs coarse to fine: both images are low-passed with a
Gaussian whose width halves at each stage (32 px at 256 px picture width
down to none), Adam on (k, l, s) with the parameters projected back into
the limits after every step; the last stage can also move the vertices.
The blur, the loss and the optimiser are PyTorch operations on the CUDA
tensors; the rendering and its adjoint are the library's kernels.
"""
from __future__ import annotations

import time

import torch

from . import vsr as V

LIMITS = {"k": (-1.0, 1.0), "l": (0.05, 1.0), "s": (0.5, 1.0)}


def gaussian_blur(img, sigma):
    """Separable Gaussian low-pass of a [H, W] tensor (replicated border)."""
    if sigma <= 0:
        return img
    rad = int(3 * sigma) + 1
    x = torch.arange(-rad, rad + 1, device=img.device, dtype=img.dtype)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    k = k / k.sum()
    im = img[None, None]
    im = torch.nn.functional.conv2d(torch.nn.functional.pad(im, (rad, rad, 0, 0), mode="replicate"),
                                    k.view(1, 1, 1, -1))
    im = torch.nn.functional.conv2d(torch.nn.functional.pad(im, (0, 0, rad, rad), mode="replicate"),
                                    k.view(1, 1, -1, 1))
    return im[0, 0]


def fit_lens(target, tris, colors, start, renderer: V.ShadedRenderer, sigmas=(32, 16, 8, 4, 2, 1, 0),
             steps=40, lr=0.01, vertex_steps=0, vertex_lr=1e-3, omega=None, callback=None):
    """Fit (k, l, s) (Omega held) so that the render of `tris` / `colors`
    matches `target` ([H, W] CUDA float32).

    start: dict with k, l, s, omega.  sigmas: blur widths in pixels at a
    256-pixel-wide picture (scaled with the renderer's width), one stage
    each of `steps` Adam steps.  vertex_steps > 0 adds a final stage that
    also refines the vertices at full resolution.  Returns a dict with the
    fitted lens, the vertices, the loss history and the wall time."""
    W = renderer.W
    scale = W / 256.0
    om = start["omega"] if omega is None else omega
    lens = torch.tensor([start["k"], start["l"], start["s"], om], dtype=torch.float64, requires_grad=True)
    verts = tris.detach().clone().requires_grad_(vertex_steps > 0)
    cols = colors.detach()
    opt = torch.optim.Adam([lens], lr=lr)
    hist = []
    t0 = time.perf_counter()

    def project():
        with torch.no_grad():
            for q, name in enumerate(("k", "l", "s")):
                lens[q].clamp_(*LIMITS[name])

    def step(sigma, params_opt):
        params_opt.zero_grad()
        img = V.render_shaded(verts, cols, lens, renderer)[0]
        loss = ((gaussian_blur(img, sigma * scale) - gaussian_blur(target, sigma * scale)) ** 2).sum()
        loss.backward()
        lens.grad[3] = 0.0  # the angle of view is held
        params_opt.step()
        project()
        rec = (float(sigma), float(loss.detach()), *[float(x) for x in lens.detach()[:3]])
        hist.append(rec)
        if callback:
            callback(rec)

    for sigma in sigmas:
        for _ in range(steps):
            step(sigma, opt)
    if vertex_steps > 0:
        opt2 = torch.optim.Adam([{"params": [lens], "lr": lr * 0.1}, {"params": [verts], "lr": vertex_lr}])
        for _ in range(vertex_steps):
            step(0, opt2)
    torch.cuda.synchronize()
    k, l, s, o = [float(x) for x in lens.detach()]
    return {"lens": {"k": k, "l": l, "s": s, "omega": o}, "verts": verts.detach(), "history": hist,
            "seconds": time.perf_counter() - t0}
