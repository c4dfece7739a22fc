"""Training step driver (Sec. 5.1): render -> image loss (1 - lambda) L1 + lambda (1 - SSIM) -> path-replay
backward -> Adam with per-parameter learning rates and an exponential decay (1 -> 0.1 of the initial rates)
-> split / prune densification, with the coarse-to-fine resolution schedule (1/4, then 1/2 from iteration
64, then full from 200).

Every step runs in the library's kernels (render, loss and its gradient, backward, Adam, gradient-norm
accumulation, densification); this module holds the tensors and the schedule. Targets are images rendered
from a synthetic ground-truth scene: the paper's datasets are not used.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np
import torch

from . import _abi
from .render import PARAM_KEYS, Renderer

#: initial learning rates per array (means, log_scales, quats, opacity_logits, sh), the 3D Gaussian
#: splatting values for a scene of extent ~10 (the paper's "bounded Adam" rates are for its own
#: parametrisation, which it does not define)
DEFAULT_LR = (1.6e-4 * 10.0, 5e-3, 1e-3, 5e-2, 2.5e-3)


def _grads_struct(d: dict, prefix=""):
    return _abi.Grads(*(d[prefix + k].data_ptr() for k in PARAM_KEYS))


def l1_ssim(renderer: Renderer, image: torch.Tensor, target: torch.Tensor, lam: float = 0.2, grad: bool = True,
            read_loss: bool = True):
    """(L, L1, SSIM) (host floats, or None if not read) and dL/dimage (or None)."""
    H, W = image.shape[0], image.shape[1]
    dl = torch.empty_like(image) if grad else None
    out = (C.c_double * 3)()
    stream = torch.cuda.current_stream(renderer.device).cuda_stream
    rc = renderer.lib.ngs_loss_l1_ssim(renderer.ctx, image.data_ptr(), target.data_ptr(), W, H, float(lam),
                                       dl.data_ptr() if grad else None, out if read_loss else None, stream)
    _abi.check(rc, renderer.ctx)
    return (tuple(out) if read_loss else None), dl


class Adam:
    """Adam state (first and second moments) for the five parameter arrays."""

    def __init__(self, params: dict, lr=DEFAULT_LR, betas=(0.9, 0.999), eps=1e-15, bounded=True):
        self.m = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}
        self.v = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}
        self.lr = tuple(float(x) for x in lr)
        self.betas, self.eps, self.bounded = betas, float(eps), bool(bounded)
        self.t = 0

    def step(self, renderer: Renderer, params: dict, grads: dict, lr_scale: float = 1.0):
        self.t += 1
        n = params["means"].shape[0]
        K = params["sh"].numel() // (3 * n) if n else 1
        deg = int(round(math.sqrt(K))) - 1
        cfg = _abi.Adam((C.c_float * 5)(*(lr * lr_scale for lr in self.lr)), self.betas[0], self.betas[1], self.eps,
                        self.t, int(self.bounded))
        stream = torch.cuda.current_stream(renderer.device).cuda_stream
        rc = renderer.lib.ngs_adam_step(renderer.ctx, n, deg, C.byref(_grads_struct(params)),
                                        C.byref(_grads_struct(grads, "d_")), C.byref(_grads_struct(self.m)),
                                        C.byref(_grads_struct(self.v)), C.byref(cfg), stream)
        _abi.check(rc, renderer.ctx)


def densify(renderer: Renderer, params: dict, adam: Adam, accum: torch.Tensor, count: torch.Tensor,
            grad_threshold: float, min_opacity: float = 0.008, min_scale: float = 1e-4, max_gaussians: int = 200_000,
            split: bool = True, prune: bool = True):
    """Split / prune (library kernels); returns the new parameter dict (the Adam state is replaced)."""
    n = params["means"].shape[0]
    K3 = params["sh"].numel() // n if n else 3
    cap = min(2 * n, max(n, max_gaussians))
    shape = {"means": (3,), "log_scales": (3,), "quats": (4,), "opacity_logits": (), "sh": tuple(params["sh"].shape[1:])}
    new_p = {k: torch.empty((cap, *shape[k]), device=params[k].device) for k in PARAM_KEYS}
    new_m = {k: torch.empty_like(new_p[k]) for k in PARAM_KEYS}
    new_v = {k: torch.empty_like(new_p[k]) for k in PARAM_KEYS}
    cfg = _abi.DensifyCfg(float(grad_threshold), float(min_opacity), float(min_scale), int(split), int(prune),
                          int(max_gaussians))
    n_out = C.c_int64()
    deg = int(round(math.sqrt(K3 // 3))) - 1
    stream = torch.cuda.current_stream(renderer.device).cuda_stream
    rc = renderer.lib.ngs_densify(renderer.ctx, n, deg, C.byref(_grads_struct(params)), C.byref(_grads_struct(adam.m)),
                                  C.byref(_grads_struct(adam.v)), accum.data_ptr(), count.data_ptr(), C.byref(cfg),
                                  cap, C.byref(_grads_struct(new_p)), C.byref(_grads_struct(new_m)),
                                  C.byref(_grads_struct(new_v)), C.byref(n_out), stream)
    _abi.check(rc, renderer.ctx)
    k = n_out.value
    adam.m = {key: new_m[key][:k].contiguous() for key in PARAM_KEYS}
    adam.v = {key: new_v[key][:k].contiguous() for key in PARAM_KEYS}
    return {key: new_p[key][:k].contiguous() for key in PARAM_KEYS}


def scaled_camera(cam: dict, factor: int) -> dict:
    """The camera at 1/factor resolution (intrinsics scaled, same pose)."""
    if factor == 1:
        return cam
    W, H = max(1, cam["width"] // factor), max(1, cam["height"] // factor)
    return dict(cam, width=W, height=H, fx=cam["fx"] / factor, fy=cam["fy"] / factor, cx=cam["cx"] / factor,
                cy=cam["cy"] / factor)


class Trainer:
    """One reconstruction run on synthetic targets (Sec. 5.1's recipe): per step one training camera,
    loss, backward, Adam; split every `densify_every` steps and prune every `prune_every` steps until
    `densify_until`; learning rates decayed exponentially from 1x to 0.1x over `iters`.

    The split criterion is the mean, over the steps where a Gaussian was visible, of |dL/dmean| with L the
    per-pixel mean loss (world units); `grad_threshold` is in those units."""

    def __init__(self, params: dict, cameras: list, targets: dict, model="sup", iters: int = 1000, lam: float = 0.2,
                 lr=DEFAULT_LR, densify_every: int = 100, prune_every: int = 200, densify_until: int = 3000,
                 grad_threshold: float = 2e-4, max_gaussians: int = 200_000, coarse_to_fine=((0, 4), (64, 2), (200, 1)),
                 options=None, renderer: Renderer | None = None, seed: int = 0):
        self.r = renderer or Renderer(params["means"].device)
        self.params = {k: params[k].clone().contiguous() for k in PARAM_KEYS}
        self.cameras, self.targets, self.model = cameras, targets, model
        self.iters, self.lam = iters, lam
        self.adam = Adam(self.params, lr)
        self.densify_every, self.prune_every, self.densify_until = densify_every, prune_every, densify_until
        self.grad_threshold, self.max_gaussians = grad_threshold, max_gaussians
        self.schedule = coarse_to_fine
        self.options = options
        self.rng = np.random.default_rng(seed)
        self.it = 0
        self._reset_accum()
        self.frames = {}

    def _reset_accum(self):
        n = self.params["means"].shape[0]
        dev = self.params["means"].device
        self.accum = torch.zeros(n, device=dev)
        self.count = torch.zeros(n, device=dev)

    def factor(self) -> int:
        f = 1
        for start, fac in self.schedule:
            if self.it >= start:
                f = fac
        return f

    def step(self, read_loss: bool = False) -> dict:
        t0 = time.perf_counter()
        f = self.factor()
        v = int(self.rng.integers(0, len(self.cameras)))
        cam = scaled_camera(self.cameras[v], f)
        key = (v, f)
        img, od, frame = self.r.render(self.params, cam, self.model, self.options, frame=self.frames.get(key))
        self.frames[key] = frame
        loss, dl = l1_ssim(self.r, img, self.targets[(v, f)], self.lam, grad=True, read_loss=read_loss)
        grads = self.r.backward(frame, self.params, dl)
        self.r.lib.ngs_accumulate_grad_norm(self.r.ctx, self.params["means"].shape[0], grads["d_means"].data_ptr(),
                                            self.accum.data_ptr(), self.count.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
        lr_scale = 0.1 ** (self.it / max(1, self.iters - 1))  # exponential decay 1 -> 0.1
        self.adam.step(self.r, self.params, grads, lr_scale)
        self.it += 1
        changed = False
        if self.it < self.densify_until and self.it % self.densify_every == 0:
            prune = self.it % self.prune_every == 0
            self.params = densify(self.r, self.params, self.adam, self.accum, self.count, self.grad_threshold,
                                  max_gaussians=self.max_gaussians, split=True, prune=prune)
            changed = True
        elif self.it < self.densify_until and self.it % self.prune_every == 0:
            self.params = densify(self.r, self.params, self.adam, self.accum, self.count, self.grad_threshold,
                                  max_gaussians=self.max_gaussians, split=False, prune=True)
            changed = True
        if changed:
            self._reset_accum()
        out = {"it": self.it, "factor": f, "view": v, "n": int(self.params["means"].shape[0]),
               "overdraw_mean": None, "wall_ms": (time.perf_counter() - t0) * 1e3}
        if loss is not None:
            out.update(loss=loss[0], l1=loss[1], ssim=loss[2], overdraw_mean=float(od.float().mean()))
        return out


def render_targets(renderer: Renderer, gt_params: dict, cameras: list, model, factors=(1, 2, 4), options=None) -> dict:
    """Targets[(view, factor)]: the ground-truth scene rendered at each resolution of the schedule."""
    out = {}
    for v, cam in enumerate(cameras):
        for f in factors:
            img, _, fr = renderer.render(gt_params, scaled_camera(cam, f), model, options)
            out[(v, f)] = img.clone()
            renderer.recycle(fr)
    return out


def psnr(renderer: Renderer, params: dict, cameras: list, targets: dict, model, options=None) -> float:
    """Mean PSNR over the training views at full resolution."""
    vals = []
    for v, cam in enumerate(cameras):
        img, _, fr = renderer.render(params, cam, model, options)
        mse = float(((img - targets[(v, 1)]) ** 2).mean())
        vals.append(10.0 * math.log10(1.0 / max(mse, 1e-12)))
        renderer.recycle(fr)
    return float(np.mean(vals))
