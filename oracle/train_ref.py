"""Training-step oracle (numpy, FP64): the image loss (1 - lambda) L1 + lambda (1 - SSIM) and its gradient,
one Adam update, and split / prune densification, each written out from its definition.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the test suite may import it.

* SSIM (Wang, Bovik, Sheikh, Simoncelli 2004) with the 11 x 11 Gaussian window of standard deviation 1.5,
  C1 = 0.01^2, C2 = 0.03^2 and zero padding ("same" output size), per channel, averaged over pixels and
  channels -- the convention of 3D Gaussian splatting, which Sec. 5.1's loss follows.
* Adam (Kingma and Ba 2015) with bias correction; "bounded": the update clipped to [-lr, lr].
* Densification (Sec. 5.1): prune when sigmoid(logit) < min_opacity or max exp(log_scale) < min_scale;
  else split when accum / count > grad_threshold; splits granted in index order up to max_gaussians; a
  split gives two children at mu +- sigma_a / 2 along the longest axis a with sigma_a * sqrt(3) / 2.
"""
from __future__ import annotations

import numpy as np

C1, C2 = 0.01 ** 2, 0.03 ** 2
RADIUS = 5


def gaussian_window(sigma: float = 1.5, radius: int = RADIUS) -> np.ndarray:
    d = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-d * d / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' correlation of each [H, W] plane of a [H, W, C] array with the separable window
    g x g (symmetric, so also its convolution and its own adjoint)."""
    r = len(g) // 2
    H, W = a.shape[:2]
    p = np.zeros((H + 2 * r, W + 2 * r) + a.shape[2:])
    p[r:r + H, r:r + W] = a
    h = sum(g[k] * p[:, k:k + W] for k in range(len(g)))
    return sum(g[k] * h[k:k + H] for k in range(len(g)))


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    g = gaussian_window()
    mx, my = blur(x, g), blur(y, g)
    vx, vy = blur(x * x, g) - mx * mx, blur(y * y, g) - my * my
    cxy = blur(x * y, g) - mx * my
    return ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))


def l1_ssim(x: np.ndarray, y: np.ndarray, lam: float = 0.2):
    """Returns (L, L1, SSIM, dL/dx) for [H, W, 3] images x (rendered) and y (target)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    g = gaussian_window()
    n = x.size
    mx, my = blur(x, g), blur(y, g)
    sxx, syy, sxy = blur(x * x, g), blur(y * y, g), blur(x * y, g)
    n1, n2 = 2 * mx * my + C1, 2 * (sxy - mx * my) + C2
    d1, d2 = mx * mx + my * my + C1, (sxx - mx * mx) + (syy - my * my) + C2
    s = n1 * n2 / (d1 * d2)
    ssim = s.mean()
    l1 = np.abs(x - y).mean()
    # chain rule through the windowed moments: s depends on x through mx, sxx and sxy
    ds_dmx = s * (2 * my / n1 - 2 * my / n2 - 2 * mx / d1 + 2 * mx / d2)
    ds_dsxx = -s / d2
    ds_dsxy = 2 * s / n2
    dssim = (blur(ds_dmx, g) + 2 * x * blur(ds_dsxx, g) + y * blur(ds_dsxy, g)) / n
    grad = (1 - lam) * np.sign(x - y) / n - lam * dssim
    return (1 - lam) * l1 + lam * (1 - ssim), l1, ssim, grad


def adam_step(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-15, bounded=True):
    """One Adam update of the arrays (p, m, v) with gradient g at step t (1-based); returns new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    step = lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    if bounded:
        step = np.clip(step, -lr, lr)
    return p - step, m, v


def _rotation_column(q, a):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return R[:, a]


def densify(params: dict, m: dict, v: dict, accum, count, grad_threshold, min_opacity, min_scale, max_gaussians,
            split=True, prune=True):
    """Returns (params, m, v) after split / prune, in index order."""
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    n = len(params["means"])
    op = 1.0 / (1.0 + np.exp(-np.asarray(params["opacity_logits"], np.float64)))
    smax = np.exp(np.asarray(params["log_scales"], np.float64).max(axis=1))
    dec = np.ones(n, np.int64)
    for i in range(n):
        if prune and (op[i] < min_opacity or smax[i] < min_scale):
            dec[i] = 0
        elif split and count[i] > 0 and accum[i] / count[i] > grad_threshold:
            dec[i] = 2
    survivors = int((dec != 0).sum())
    allowed = min(int((dec == 2).sum()), max(0, max_gaussians - survivors))
    out = {k: [] for k in keys}
    om = {k: [] for k in keys}
    ov = {k: [] for k in keys}
    granted = 0
    for i in range(n):
        if dec[i] == 0:
            continue
        if dec[i] == 2 and granted < allowed:
            granted += 1
            ls = np.asarray(params["log_scales"][i], np.float64)
            a = _first_max(ls)
            r = _rotation_column(params["quats"][i], a)
            half = 0.5 * np.exp(ls[a])
            for sgn in (1.0, -1.0):
                for k in keys:
                    val = np.array(params[k][i], np.float64, copy=True)
                    if k == "means":
                        val = val + sgn * half * r
                    if k == "log_scales":
                        val[a] += np.log(np.sqrt(3.0) / 2.0)
                    out[k].append(val)
                    om[k].append(np.zeros_like(val))
                    ov[k].append(np.zeros_like(val))
            continue
        for k in keys:
            out[k].append(np.array(params[k][i], np.float64))
            om[k].append(np.array(m[k][i], np.float64))
            ov[k].append(np.array(v[k][i], np.float64))
    pack = lambda d: {k: np.array(d[k]) for k in keys}  # noqa: E731
    return pack(out), pack(om), pack(ov)


def _first_max(ls):
    """Index of the largest entry, the first among equals (the kernel's comparison order)."""
    if ls[0] >= ls[1]:
        return 0 if ls[0] >= ls[2] else 2
    return 1 if ls[1] >= ls[2] else 2
