"""ctypes mirror of include/ngs.h (argument marshalling only).

Loading fails loudly when the CUDA library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

NGS_OK = 0
NGS_ERR_INVALID_ARG = -1
NGS_ERR_OUT_OF_MEMORY = -2
NGS_ERR_CUDA = -3
NGS_ERR_DEVICE_CHECK = -5
NGS_ERR_CAPACITY = -6
NGS_MODEL_EXP = 0
NGS_MODEL_QUAD = 1
NGS_MODEL_BLEND = 2
NGS_MODEL_VICINI = 3
NGS_SCHEDULE_TILES = 0
NGS_SCHEDULE_PERSISTENT = 1
NGS_NUM_STAGES = 8
NGS_PEAK_FFMA = 0
NGS_PEAK_FFMA2 = 1
NGS_PEAK_EX2 = 2
STAGES = ("project", "depth_sort", "scan_emit", "tile_sort", "tile_ranges", "composite_fwd", "composite_bwd",
          "project_bwd")


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("param", C.c_float)]


class Options(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_eps", C.c_float), ("dilation", C.c_float),
                ("near_plane", C.c_float), ("background", C.c_float * 3), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("max_splats", C.c_int32), ("chunk", C.c_int32), ("schedule", C.c_int32)]


class TuneEntry(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("chunk", C.c_int32), ("schedule", C.c_int32),
                ("ms", C.c_float)]


class Grads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p)]


class Adam(C.Structure):
    _fields_ = [("lr", C.c_float * 5), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("bounded", C.c_int32)]


class DensifyCfg(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("min_opacity", C.c_float), ("min_scale", C.c_float),
                ("split", C.c_int32), ("prune", C.c_int32), ("max_gaussians", C.c_int64)]


class FrameView(C.Structure):
    _fields_ = [("n_gaussians", C.c_int64), ("n_pairs", C.c_int64), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("log2_alpha_min", C.c_float), ("n_views", C.c_int32),
                ("records", C.c_void_p), ("keys", C.c_void_p),
                ("values", C.c_void_p), ("ranges", C.c_void_p), ("pixel_state", C.c_void_p),
                ("view_pixel_base", C.c_void_p), ("view_tile_base", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_batch_views", C.c_int32), ("mem_budget", C.c_int64),
                ("graphs", C.c_int32), ("reserved", C.c_int32), ("options", Options)]


class Request(C.Structure):
    _fields_ = [("scene", C.c_int32), ("model", Model), ("camera", Camera), ("image", C.c_void_p),
                ("overdraw", C.c_void_p), ("tag", C.c_int64)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_int64), ("status", C.c_int32), ("batch_views", C.c_int32), ("submit_s", C.c_double),
                ("start_s", C.c_double), ("done_s", C.c_double), ("pairs", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("max_batch_views", C.c_int64), ("over_budget_admissions", C.c_int64),
                ("peak_reserved_bytes", C.c_int64), ("reserved_bytes", C.c_int64), ("pending", C.c_int64),
                ("now_s", C.c_double)]


class Workspace(C.Structure):
    _fields_ = [("frame_fixed", C.c_size_t), ("frame_pairs", C.c_size_t), ("context", C.c_size_t),
                ("backward", C.c_size_t), ("total", C.c_size_t)]


#: every function declared in include/ngs.h, with its ctypes signature
SIGNATURES = {
    "ngs_default_options": (None, [C.POINTER(Options)]),
    "ngs_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "ngs_destroy": (None, [C.c_void_p]),
    "ngs_last_error": (C.c_char_p, [C.c_void_p]),
    "ngs_frame_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "ngs_frame_destroy": (None, [C.c_void_p]),
    "ngs_frame_set_async": (C.c_int, [C.c_void_p, C.c_int]),
    "ngs_frame_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "ngs_render": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.POINTER(Model),
                             C.POINTER(Options), C.c_void_p, C.c_void_p, C.c_void_p]),
    "ngs_render_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32,
                                   C.POINTER(Model), C.POINTER(Options), C.c_void_p, C.c_void_p, C.c_void_p]),
    "ngs_render_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.c_void_p, C.POINTER(Grads),
                                      C.c_void_p]),
    "ngs_render_backward_static": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.c_void_p,
                                             C.POINTER(Grads), C.c_void_p]),
    "ngs_frame_view_get": (C.c_int, [C.c_void_p, C.POINTER(FrameView)]),
    "ngs_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32,
                               C.POINTER(Model), C.POINTER(Options), C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(Grads), C.c_int32, C.c_int64, C.POINTER(Options), C.POINTER(TuneEntry),
                               C.c_int32, C.c_void_p]),
    "ngs_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "ngs_graph_captures": (C.c_int64, [C.c_void_p]),
    "ngs_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "ngs_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "ngs_reset_stage_times": (None, [C.c_void_p]),
    "ngs_launch_count": (C.c_int64, [C.c_void_p]),
    "ngs_workspace_bytes": (C.c_int, [C.c_int64, C.POINTER(Camera), C.c_int32, C.POINTER(Options), C.c_int64,
                                      C.POINTER(Workspace)]),
    "ngs_memory_usage": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "ngs_set_checked": (C.c_int, [C.c_void_p, C.c_int]),
    "ngs_measure_peak": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_double), C.c_void_p]),
    "ngs_loss_l1_ssim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_void_p,
                                   C.POINTER(C.c_double), C.c_void_p]),
    "ngs_adam_step": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(Grads), C.POINTER(Grads), C.POINTER(Grads),
                                C.POINTER(Grads), C.POINTER(Adam), C.c_void_p]),
    "ngs_accumulate_grad_norm": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ngs_densify": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(Grads), C.POINTER(Grads), C.POINTER(Grads),
                              C.c_void_p, C.c_void_p, C.POINTER(DensifyCfg), C.c_int64, C.POINTER(Grads),
                              C.POINTER(Grads), C.POINTER(Grads), C.POINTER(C.c_int64), C.c_void_p]),
    "ngs_default_server_config": (None, [C.POINTER(ServerConfig)]),
    "ngs_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]),
    "ngs_server_add_scene": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(C.c_int32)]),
    "ngs_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request)]),
    "ngs_server_poll": (C.c_int, [C.c_void_p, C.POINTER(Completion), C.c_int32, C.c_int32]),
    "ngs_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "ngs_server_last_error": (C.c_char_p, [C.c_void_p]),
    "ngs_server_destroy": (None, [C.c_void_p]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the built library (raises if it is missing: call paper_2603_02887_gb300.build.build())."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path} missing); run paper_2603_02887_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class NGSError(RuntimeError):
    def __init__(self, msg: str, code: int = 0):
        super().__init__(msg)
        self.code = code


class CapacityExceeded(NGSError):
    """An asynchronous render met more pairs than its frame's capacity (which has now grown): render again."""


def check(rc: int, ctx) -> None:
    if rc != NGS_OK:
        msg = load().ngs_last_error(ctx)
        cls = CapacityExceeded if rc == NGS_ERR_CAPACITY else NGSError
        raise cls(f"ngs error {rc}: {msg.decode() if msg else ''}", rc)
