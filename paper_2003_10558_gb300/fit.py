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

Checkpoints: `LensFit.state_dict()` holds everything the next step depends
on -- lens, vertices, both optimisers' moments, stage, step and the loss
history -- and `LensFit.load_state_dict()` / `load()` restore it, so a fit
stopped after any step continues where it stopped.  The lens stages are
deterministic (the lens gradient is reduced per pixel and then in a fixed
order in double precision; the blur is two matrix products), so a resumed
lens stage repeats the uninterrupted run bit for bit.  In the vertex stage the per-triangle
gradients are summed with floating-point atomics, whose order varies from
run to run: its steps agree with an uninterrupted run to rounding, as two
uninterrupted runs agree with each other.
"""
from __future__ import annotations

import copy
import time

import torch

from . import vsr as V

LIMITS = {"k": (-1.0, 1.0), "l": (0.05, 1.0), "s": (0.5, 1.0)}


_BAND = {}


def _band(n, sigma, device, dtype):
    """[n, n] matrix of the 1D Gaussian low-pass with a replicated border:
    row i holds the weights of the taps i-rad .. i+rad, clamped into [0, n)."""
    key = (n, float(sigma), str(device), dtype)
    if key not in _BAND:
        rad = int(3 * sigma) + 1
        x = torch.arange(-rad, rad + 1, dtype=torch.float64)
        w = torch.exp(-0.5 * (x / sigma) ** 2)
        w = w / w.sum()
        A = torch.zeros((n, n), dtype=torch.float64)
        rows = torch.arange(n)
        for q in range(2 * rad + 1):
            A.index_put_((rows, (rows + q - rad).clamp(0, n - 1)), w[q].expand(n), accumulate=True)
        _BAND[key] = A.to(device=device, dtype=dtype)
    return _BAND[key]


def gaussian_blur(img, sigma):
    """Separable Gaussian low-pass of a [H, W] tensor (replicated border), as
    two band-matrix products: deterministic in value and in gradient."""
    if sigma <= 0:
        return img
    H, W = img.shape
    return _band(H, sigma, img.device, img.dtype) @ img @ _band(W, sigma, img.device, img.dtype).T


class LensFit:
    """A resumable coarse-to-fine lens fit.

    target: [H, W] CUDA float32 image; tris [T, 3, 3] and colors [T] CUDA
    float32; start: dict with k, l, s, omega; renderer: a ShadedRenderer of
    the target's size.  sigmas: blur widths in pixels at a 256-pixel-wide
    picture (scaled with the renderer's width), one stage each of `steps`
    Adam steps on (k, l, s); vertex_steps > 0 adds a final stage that also
    refines the vertices at full resolution (the lens at a tenth of lr)."""

    def __init__(self, target, tris, colors, start, renderer: V.ShadedRenderer, sigmas=(32, 16, 8, 4, 2, 1, 0),
                 steps=40, lr=0.01, vertex_steps=0, vertex_lr=1e-3, omega=None):
        self.target = target
        self.renderer = renderer
        self.sigmas = tuple(float(s) for s in sigmas)
        self.steps = int(steps)
        self.vertex_steps = int(vertex_steps)
        self.scale = renderer.W / 256.0
        om = start["omega"] if omega is None else omega
        self.lens = torch.tensor([start["k"], start["l"], start["s"], om], dtype=torch.float64, requires_grad=True)
        self.verts = tris.detach().clone().requires_grad_(self.vertex_steps > 0)
        self.cols = colors.detach()
        self.opt = torch.optim.Adam([self.lens], lr=lr)
        self.opt2 = torch.optim.Adam([{"params": [self.lens], "lr": lr * 0.1},
                                      {"params": [self.verts], "lr": vertex_lr}]) if self.vertex_steps > 0 else None
        self.stage = 0      # index into sigmas; len(sigmas) = the vertex stage
        self.step_in_stage = 0
        self.history = []   # (sigma, loss, k, l, s) per step
        self.seconds = 0.0
        self._blurred = {}

    # -- progress ---------------------------------------------------------
    def n_stages(self):
        return len(self.sigmas) + (1 if self.vertex_steps > 0 else 0)

    def done(self):
        return self.stage >= self.n_stages()

    def _stage_len(self, stage):
        return self.steps if stage < len(self.sigmas) else self.vertex_steps

    def _target_blurred(self, sigma):
        if sigma not in self._blurred:
            self._blurred[sigma] = gaussian_blur(self.target, sigma * self.scale)
        return self._blurred[sigma]

    def step(self):
        """One Adam step of the current stage; returns its history record."""
        vertex = self.stage >= len(self.sigmas)
        sigma = 0.0 if vertex else self.sigmas[self.stage]
        opt = self.opt2 if vertex else self.opt
        opt.zero_grad()
        img = V.render_shaded(self.verts, self.cols, self.lens, self.renderer)[0]
        loss = ((gaussian_blur(img, sigma * self.scale) - self._target_blurred(sigma)) ** 2).sum()
        loss.backward()
        self.lens.grad[3] = 0.0  # the angle of view is held
        opt.step()
        with torch.no_grad():
            for q, name in enumerate(("k", "l", "s")):
                self.lens[q].clamp_(*LIMITS[name])
        rec = (sigma, float(loss.detach()), *[float(x) for x in self.lens.detach()[:3]])
        self.history.append(rec)
        self.step_in_stage += 1
        if self.step_in_stage >= self._stage_len(self.stage):
            self.stage += 1
            self.step_in_stage = 0
        return rec

    def run(self, max_steps=None, callback=None):
        """Run until the fit is done or max_steps more steps have run."""
        t0 = time.perf_counter()
        n = 0
        while not self.done() and (max_steps is None or n < max_steps):
            rec = self.step()
            n += 1
            if callback:
                callback(rec)
        torch.cuda.synchronize()
        self.seconds += time.perf_counter() - t0
        return self

    def result(self):
        k, l, s, o = [float(x) for x in self.lens.detach()]
        return {"lens": {"k": k, "l": l, "s": s, "omega": o}, "verts": self.verts.detach(),
                "history": list(self.history), "seconds": self.seconds}

    # -- checkpoints ------------------------------------------------------
    def state_dict(self):
        """Everything the next step depends on (tensors copied to the host)."""
        return {"lens": self.lens.detach().cpu().clone(), "verts": self.verts.detach().cpu().clone(),
                "opt": copy.deepcopy(self.opt.state_dict()),
                "opt2": copy.deepcopy(self.opt2.state_dict()) if self.opt2 is not None else None,
                "stage": self.stage, "step_in_stage": self.step_in_stage, "history": list(self.history),
                "sigmas": self.sigmas, "steps": self.steps, "vertex_steps": self.vertex_steps,
                "seconds": self.seconds}

    def load_state_dict(self, sd):
        if (tuple(sd["sigmas"]) != self.sigmas or sd["steps"] != self.steps
                or sd["vertex_steps"] != self.vertex_steps):
            raise ValueError("checkpoint of a fit with another schedule")
        with torch.no_grad():
            self.lens.copy_(sd["lens"].to(self.lens.device))
            self.verts.copy_(sd["verts"].to(self.verts.device))
        self.opt.load_state_dict(sd["opt"])
        if self.opt2 is not None:
            self.opt2.load_state_dict(sd["opt2"])
        self.stage = int(sd["stage"])
        self.step_in_stage = int(sd["step_in_stage"])
        self.history = list(sd["history"])
        self.seconds = float(sd["seconds"])
        return self

    def save(self, path):
        torch.save(self.state_dict(), path)

    def load(self, path):
        return self.load_state_dict(torch.load(path, map_location="cpu", weights_only=False))


def fit_lens(target, tris, colors, start, renderer: V.ShadedRenderer, sigmas=(32, 16, 8, 4, 2, 1, 0),
             steps=40, lr=0.01, vertex_steps=0, vertex_lr=1e-3, omega=None, callback=None):
    """Fit (k, l, s) (Omega held) so that the render of `tris` / `colors`
    matches `target` ([H, W] CUDA float32); see LensFit.  Returns a dict
    with the fitted lens, the vertices, the loss history and the wall time."""
    f = LensFit(target, tris, colors, start, renderer, sigmas=sigmas, steps=steps, lr=lr, vertex_steps=vertex_steps,
                vertex_lr=vertex_lr, omega=omega)
    return f.run(callback=callback).result()
