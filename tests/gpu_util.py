"""Helpers for the GPU tests: device views of library buffers, parameter upload, comparisons."""
import numpy as np
import torch

from paper_2603_02887_gb300.render import PARAM_KEYS


class _DevArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def device_array(ptr, shape, dtype):
    """Copy a library-owned device buffer to a numpy array."""
    typestr = {np.float32: "<f4", np.uint64: "<u8", np.uint32: "<u4", np.int32: "<i4"}[dtype]
    if int(np.prod(shape)) == 0:
        return np.zeros(shape, dtype)
    t = torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")
    return t.cpu().numpy().copy()


def upload(scene, device="cuda"):
    return {k: torch.from_numpy(np.ascontiguousarray(scene[k])).to(device) for k in PARAM_KEYS}


def frame_arrays(frame):
    v = frame.view()
    n, P = v["n_gaussians"], v["n_pairs"]
    T = v["tiles_x"] * v["tiles_y"]
    return dict(
        records=device_array(v["records"], (n, 12), np.float32),
        keys=device_array(v["keys"], (P,), np.uint64),
        values=device_array(v["values"], (P,), np.uint32),
        ranges=device_array(v["ranges"], (T, 2), np.uint32),
        state=device_array(v["pixel_state"], (v["height"], v["width"], 8), np.float32),
        view=v,
    )


def grad_mismatch(gpu, ref, rel=1e-3, exclude=None, scale=None, scale_rel=1e-4):
    """Elements violating |g - g_ref| <= rel * max(|g_ref|, 1e-3 * max|g_ref|) + scale_rel * scale, per tensor.

    ``scale`` is the oracle's error scale of each gradient (sum of absolute per-pixel terms through the
    absolute Jacobian). A gradient that is a sum of terms that cancel can only be as accurate as its
    largest terms: in FP32 each term carries the error of the O(1) running quantities the replay
    differences (1 - S at the saturating splat, L0 - sum E pbar, A - E_k taubar_k), about n u ~ 1e-5
    absolute for lists of n ~ 100 splats, i.e. up to ~1e-4 of the term's size. A wrong term is off by
    O(scale).
    """
    a = np.asarray(gpu, np.float64).reshape(len(ref), -1)
    b = np.asarray(ref, np.float64).reshape(len(ref), -1)
    floor = 1e-3 * np.abs(b).max() if b.size else 0.0
    tol = rel * np.maximum(np.abs(b), floor)
    if scale is not None:
        tol = tol + scale_rel * np.asarray(scale, np.float64).reshape(len(ref), -1)
    bad = np.abs(a - b) > tol
    if exclude is not None:
        bad[exclude] = False
    return bad


def describe_mismatch(gpu, ref, bad, scale=None, limit=5):
    a = np.asarray(gpu, np.float64).reshape(len(ref), -1)
    b = np.asarray(ref, np.float64).reshape(len(ref), -1)
    s = None if scale is None else np.asarray(scale, np.float64).reshape(len(ref), -1)
    out = []
    for gi, j in list(zip(*np.nonzero(bad)))[:limit]:
        out.append(f"[{gi},{j}] gpu={a[gi, j]:.6g} ref={b[gi, j]:.6g}" + ("" if s is None else f" scale={s[gi, j]:.4g}"))
    return "; ".join(out)


def batch_arrays(frame):
    """Host copies of a (batch) frame's buffers: records [n_views n, 12], keys, values, ranges [tiles, 2],
    replay state [pixels, 8], and the per-view pixel / tile bases."""
    v = frame.view()
    n, P, m = v["n_gaussians"], v["n_pairs"], v["n_views"]
    T = int(v["view_tile_base"][m])
    npix = int(v["view_pixel_base"][m])
    return dict(
        records=device_array(v["records"], (m * n, 12), np.float32),
        keys=device_array(v["keys"], (P,), np.uint64),
        values=device_array(v["values"], (P,), np.uint32),
        ranges=device_array(v["ranges"], (T, 2), np.uint32),
        state=device_array(v["pixel_state"], (npix, 8), np.float32),
        pixel_base=v["view_pixel_base"], tile_base=v["view_tile_base"], view=v,
    )
