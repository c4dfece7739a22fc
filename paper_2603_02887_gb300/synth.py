"""Seeded synthetic inputs: Gaussian scenes, cameras and upstream gradients.

This module holds no arithmetic of the rendering method; it only draws parameters. Both the CUDA
path and the FP64 oracle are fed from it. All arrays are float32 numpy arrays (the parameter layout
of the C ABI: means[N,3], log_scales[N,3], quats[N,4] (w,x,y,z, not normalised), opacity_logits[N],
sh[N,(d+1)^2,3]).

Scene recipes (stand-ins for the paper's captures, which are not available here):

* ``tiny_scene``: N = 1000, means uniform in [-1,1]^2 x [2,6], log-scales ~ N(-3, 0.5), random unit
  quaternions, opacity = sigmoid(N(0,1)), RGB uniform in [0,1] as SH degree 0.
* ``clustered_scene``: a mixture of 64 anisotropic clusters; centres uniform in a 10 m box around the
  origin, per-cluster covariance Q diag(lambda) Q^T with Q random orthogonal and lambda log-uniform in
  [0.05, 2] m^2; log-scales ~ N(-4, 0.7), opacity logits ~ N(0.5, 1.5), SH degree 3 with the colour
  term uniform in [0,1] and the higher bands ~ N(0, 0.1). At ~0.5-3.4M primitives this is the size of
  the paper's refinement scenes; the exponential overdraw it produces lands in the range the paper
  reports for them.
"""
from __future__ import annotations

import math
import numpy as np

#: Reciprocal of the constant degree-0 real spherical harmonic 1/(2 sqrt(pi)); used only to draw an SH
#: colour coefficient that decodes to a chosen RGB value.
_INV_Y00 = 2.0 * math.sqrt(math.pi)


def _rgb_to_dc(rgb):
    return ((rgb - 0.5) * _INV_Y00).astype(np.float32)


def _random_unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def tiny_scene(seed: int = 0, n: int = 1000):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 6, n)], axis=1)
    scene = dict(
        means=means.astype(np.float32),
        log_scales=rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32),
        quats=_random_unit_quats(rng, n),
        opacity_logits=rng.normal(0.0, 1.0, n).astype(np.float32),
        sh=_rgb_to_dc(rng.uniform(0, 1, (n, 1, 3))),
    )
    return scene


def clustered_scene(n: int, seed: int = 0, sh_degree: int = 3, clusters: int = 64, box: float = 10.0):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-box / 2, box / 2, (clusters, 3))
    Qs = []
    for _ in range(clusters):
        Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
        Qs.append(Q * np.sign(np.diag(R)))
    lam = np.exp(rng.uniform(math.log(0.05), math.log(2.0), (clusters, 3)))
    which = rng.integers(0, clusters, n)
    local = rng.standard_normal((n, 3)) * np.sqrt(lam[which])
    means = centres[which] + np.einsum("nij,nj->ni", np.stack(Qs)[which], local)
    K = (sh_degree + 1) ** 2
    sh = np.empty((n, K, 3), dtype=np.float32)
    sh[:, 0, :] = _rgb_to_dc(rng.uniform(0, 1, (n, 3)))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    return dict(
        means=means.astype(np.float32),
        log_scales=rng.normal(-4.0, 0.7, (n, 3)).astype(np.float32),
        quats=_random_unit_quats(rng, n),
        opacity_logits=rng.normal(0.5, 1.5, n).astype(np.float32),
        sh=sh,
    )


def perturbed(scene, seed: int, sigma: float = 0.01):
    """Copy of ``scene`` with N(0, sigma) noise added to every parameter array."""
    rng = np.random.default_rng(seed)
    return {k: (v + rng.normal(0.0, sigma, v.shape)).astype(np.float32) for k, v in scene.items()}


def pinhole(viewmat, width: int, height: int, fx: float, fy: float, cx=None, cy=None):
    return dict(viewmat=np.asarray(viewmat, dtype=np.float32).reshape(3, 4), width=int(width), height=int(height),
                fx=float(fx), fy=float(fy), cx=float(width / 2 if cx is None else cx),
                cy=float(height / 2 if cy is None else cy))


def tiny_camera():
    """Camera at the origin looking down +z, 128 x 128 px, fx = fy = 150."""
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return pinhole(vm, 128, 128, 150.0, 150.0)


def look_at(eye, target, width: int, height: int, hfov_deg: float = 60.0):
    """World->view [R|t] for a camera at ``eye`` looking at ``target`` (+z forward, +y down in the image)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    down_hint = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.99 else np.array([0.0, 0.0, 1.0])
    x = np.cross(down_hint, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    focal = width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
    return pinhole(np.concatenate([R, t[:, None]], axis=1), width, height, focal, focal)


def outside_camera(width: int = 1920, height: int = 1080, distance: float = 15.0):
    """Camera outside the 10 m box, ``distance`` from its centre, looking at it, 60 deg horizontal FOV."""
    d = np.array([0.25, -0.2, -1.0])
    eye = distance * d / np.linalg.norm(d)
    return look_at(eye, np.zeros(3), width, height)


RESOLUTIONS = ((640, 360), (1280, 720), (1297, 840), (1920, 1080))


def orbit_cameras(count: int, radius: float = 12.0, seed: int = 2, resolutions=RESOLUTIONS):
    """``count`` cameras with poses uniform on a sphere of ``radius`` around the origin, each looking at it,
    with a resolution drawn uniformly from ``resolutions``."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(count):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        w, h = resolutions[rng.integers(0, len(resolutions))]
        cams.append(look_at(radius * v, np.zeros(3), w, h))
    return cams


def upstream_gradient(height: int, width: int, seed: int = 3):
    """A dense dL/dimage [H, W, 3] with entries +-1 (the gradient of an L1 loss) drawn at random."""
    rng = np.random.default_rng(seed)
    return np.sign(rng.standard_normal((height, width, 3))).astype(np.float32)
