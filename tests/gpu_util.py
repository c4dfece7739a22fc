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
