"""PyTorch-facing API over the C ABI: ``Renderer`` (contexts and frames), and ``render`` as a
``torch.autograd.Function`` whose backward is the library's path-replay adjoint.

PyTorch only provides device memory and the current stream; every step of rendering and of its
gradient runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np
import torch

from . import _abi

#: model name -> (kind, parameter): exponential, and the quadratic mother transmittance with
#: c = -0.5 (sub-linear), 0 (linear), +0.5 (super-linear) as in the paper's experiments (Sec. 5)
MODELS = {"exp": (_abi.NGS_MODEL_EXP, 0.0), "sub": (_abi.NGS_MODEL_QUAD, -0.5), "lin": (_abi.NGS_MODEL_QUAD, 0.0),
          "sup": (_abi.NGS_MODEL_QUAD, 0.5)}
#: the other rows of Table 1 on the same kernels, with the parameter of the paper's figures (gamma = 0.5)
EXTRA_MODELS = {"blend": (_abi.NGS_MODEL_BLEND, 0.5), "vicini": (_abi.NGS_MODEL_VICINI, 0.5)}
KINDS = {"exp": _abi.NGS_MODEL_EXP, "quad": _abi.NGS_MODEL_QUAD, "blend": _abi.NGS_MODEL_BLEND,
         "vicini": _abi.NGS_MODEL_VICINI}
PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def model_spec(model):
    """A model name ("exp", "sub", "lin", "sup", "blend", "vicini") or a (kind, parameter) pair, kind a
    name of KINDS or its number; returns (kind number, parameter)."""
    if isinstance(model, str):
        return MODELS[model] if model in MODELS else EXTRA_MODELS[model]
    kind, param = model
    if isinstance(kind, str):
        kind = KINDS[kind]
    return int(kind), float(param)


def default_options(**overrides) -> dict:
    o = _abi.Options()
    _abi.load().ngs_default_options(C.byref(o))
    d = dict(alpha_min=o.alpha_min, alpha_max=o.alpha_max, t_eps=o.t_eps, dilation=o.dilation,
             near_plane=o.near_plane, background=tuple(o.background), tile_w=o.tile_w, tile_h=o.tile_h,
             max_splats=o.max_splats, chunk=o.chunk, schedule=o.schedule)
    d.update(overrides)
    return d


def _options(opts) -> _abi.Options:
    d = default_options(**(opts or {}))
    o = _abi.Options()
    for k in ("alpha_min", "alpha_max", "t_eps", "dilation", "near_plane"):
        setattr(o, k, float(d[k]))
    for i in range(3):
        o.background[i] = float(d["background"][i])
    o.tile_w, o.tile_h, o.max_splats = int(d["tile_w"]), int(d["tile_h"]), int(d["max_splats"])
    sched = d["schedule"]
    if isinstance(sched, str):
        sched = {"tiles": _abi.NGS_SCHEDULE_TILES, "persistent": _abi.NGS_SCHEDULE_PERSISTENT}[sched]
    o.chunk, o.schedule = int(d["chunk"]), int(sched)
    return o


def _camera(cam) -> _abi.Camera:
    c = _abi.Camera()
    vm = np.asarray(cam["viewmat"], dtype=np.float32).reshape(12)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def _check_param(t: torch.Tensor, name: str, device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    return t.contiguous()


def _gaussians(params: dict, device=None):
    ts = {k: _check_param(params[k], k, device) for k in PARAM_KEYS}
    n = ts["means"].shape[0]
    if n > 0:
        K = ts["sh"].numel() // (3 * n)
    else:
        K = ts["sh"].shape[1] if ts["sh"].dim() == 3 else 1
    deg = int(round(K ** 0.5)) - 1
    if (deg + 1) ** 2 != K or deg > 3:
        raise ValueError("sh must have (d+1)^2 coefficients per Gaussian, d <= 3")
    expect = {"means": n * 3, "log_scales": n * 3, "quats": n * 4, "opacity_logits": n, "sh": n * K * 3}
    for k, m in expect.items():
        if ts[k].numel() != m:
            raise ValueError(f"{k} has {ts[k].numel()} elements, expected {m}")
    g = _abi.Gaussians(n, deg, *(ts[k].data_ptr() for k in PARAM_KEYS))
    return g, ts


class Frame:
    """Replay state of one render (owned by the library, reused across renders)."""

    def __init__(self, renderer: "Renderer"):
        self.renderer = renderer
        self.handle = C.c_void_p()
        _abi.check(_abi.load().ngs_frame_create(renderer.ctx, C.byref(self.handle)), renderer.ctx)
        self.width = self.height = 0
        self.n_pixels = 0
        self.sizes = []  # (height, width) per view of the last render

    def view(self) -> dict:
        """The frame's buffers: device pointers, plus the per-view pixel and tile bases as numpy arrays."""
        v = _abi.FrameView()
        _abi.check(_abi.load().ngs_frame_view_get(self.handle, C.byref(v)), self.renderer.ctx)
        d = {f: getattr(v, f) for f, _ in _abi.FrameView._fields_}
        m = d["n_views"]
        d["view_pixel_base"] = np.ctypeslib.as_array((C.c_int64 * (m + 1)).from_address(d["view_pixel_base"])).copy()
        d["view_tile_base"] = np.ctypeslib.as_array((C.c_uint32 * (m + 1)).from_address(d["view_tile_base"])).copy()
        return d

    def split(self, packed: torch.Tensor) -> list:
        """Per-view views [H_v, W_v, ...] of a tensor packed like the last render's images."""
        out, base = [], 0
        for h, w in self.sizes:
            out.append(packed[base:base + h * w].view(h, w, *packed.shape[1:]))
            base += h * w
        return out

    def set_async(self, enable: bool = True):
        """Asynchronous renders into this frame (no host synchronisation after binning; ngs_frame_set_async)."""
        _abi.check(_abi.load().ngs_frame_set_async(self.handle, int(bool(enable))), self.renderer.ctx)

    def status(self) -> int:
        """Wait for the frame's last render; return its pair count. Raises _abi.CapacityExceeded if an
        asynchronous render since the last call met more pairs than the frame's capacity (then render again),
        _abi.NGSError for other errors (ngs_frame_status)."""
        n = C.c_int64()
        _abi.check(_abi.load().ngs_frame_status(self.handle, C.byref(n)), self.renderer.ctx)
        return int(n.value)

    def release(self):
        if self.handle:
            _abi.load().ngs_frame_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Renderer:
    """One library context on one CUDA device. Not thread-safe; use one per thread."""

    def __init__(self, device=None):
        self.lib = _abi.load()
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        with torch.cuda.device(self.device):
            self.ctx = C.c_void_p()
            _abi.check(self.lib.ngs_create(C.byref(self.ctx)), None)
        self._pool = []

    def close(self):
        for f in self._pool:
            f.release()
        self._pool = []
        if self.ctx:
            self.lib.ngs_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # frames -------------------------------------------------------------------------------------
    def frame(self) -> Frame:
        return self._pool.pop() if self._pool else Frame(self)

    def recycle(self, frame: Frame):
        frame.set_async(False)
        self._pool.append(frame)

    # calls --------------------------------------------------------------------------------------
    def render(self, params: dict, camera: dict, model="sup", options=None, frame: Frame | None = None,
               image: torch.Tensor | None = None, overdraw: torch.Tensor | None = None):
        """Render ``params`` through ``camera``. Returns (image [H,W,3] f32, overdraw [H,W] i32, frame)."""
        g, keep = _gaussians(params, self.device)
        cam = _camera(camera)
        kind, param = model_spec(model)
        m = _abi.Model(kind, param)
        o = _options(options)
        H, W = cam.height, cam.width
        if image is None:
            image = torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        if overdraw is None:
            overdraw = torch.empty((H, W), dtype=torch.int32, device=self.device)
        frame = frame or self.frame()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self.lib.ngs_render(self.ctx, frame.handle, C.byref(g), C.byref(cam), C.byref(m), C.byref(o),
                                 image.data_ptr(), overdraw.data_ptr(), stream)
        _abi.check(rc, self.ctx)
        frame.width, frame.height, frame.n_pixels, frame.sizes = W, H, H * W, [(H, W)]
        del keep
        return image, overdraw, frame

    def render_batch(self, params: dict, cameras: list, model="sup", options=None, frame: Frame | None = None,
                     images: torch.Tensor | None = None, overdraw: torch.Tensor | None = None):
        """Render ``params`` from all ``cameras`` (any sizes) in one pass of the pipeline. Returns (images
        [sum H W, 3], overdraw [sum H W], frame), the views packed one after the other (``frame.split``
        gives per-view [H, W, ...] views). Each view equals ``render`` of its camera alone, bit for bit."""
        if len(cameras) == 0:
            raise ValueError("no cameras")
        g, keep = _gaussians(params, self.device)
        cams = (_abi.Camera * len(cameras))(*(_camera(c) for c in cameras))
        kind, param = model_spec(model)
        m = _abi.Model(kind, param)
        o = _options(options)
        sizes = [(c.height, c.width) for c in cams]
        npix = sum(h * w for h, w in sizes)
        if images is None:
            images = torch.empty((npix, 3), dtype=torch.float32, device=self.device)
        if overdraw is None:
            overdraw = torch.empty((npix,), dtype=torch.int32, device=self.device)
        if images.numel() != 3 * npix or overdraw.numel() != npix:
            raise ValueError("images / overdraw do not hold the packed pixels of all views")
        frame = frame or self.frame()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self.lib.ngs_render_batch(self.ctx, frame.handle, C.byref(g), cams, len(cameras), C.byref(m),
                                       C.byref(o), images.data_ptr(), overdraw.data_ptr(), stream)
        _abi.check(rc, self.ctx)
        frame.width, frame.height = sizes[0][1], sizes[0][0]
        frame.n_pixels, frame.sizes = npix, sizes
        del keep
        return images, overdraw, frame

    def autotune(self, params: dict, cameras: list, model="sup", options=None, backward: bool = True, reps: int = 3,
                 frame: Frame | None = None, flush_bytes: int = 256 << 20):
        """Time every tile shape x chunk x schedule on this batch (render, and backward with a unit upstream
        gradient when ``backward``; L2 cleared before each timed call when ``flush_bytes``) and return
        (fastest options dict, [(tile_w, tile_h, chunk, schedule, ms)])."""
        g, keep = _gaussians(params, self.device)
        cams = (_abi.Camera * len(cameras))(*(_camera(c) for c in cameras))
        kind, param = model_spec(model)
        m = _abi.Model(kind, param)
        o = _options(options)
        npix = sum(c.height * c.width for c in cams)
        images = torch.empty((npix, 3), dtype=torch.float32, device=self.device)
        overdraw = torch.empty((npix,), dtype=torch.int32, device=self.device)
        dl = grads = None
        if backward:
            dl = torch.ones_like(images)
            gout = {"d_" + k: torch.empty_like(keep[k]) for k in PARAM_KEYS}
            grads = _abi.Grads(*(gout["d_" + k].data_ptr() for k in PARAM_KEYS))
        frame = frame or self.frame()
        best = _abi.Options()
        table = (_abi.TuneEntry * 32)()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self.lib.ngs_autotune(self.ctx, frame.handle, C.byref(g), cams, len(cameras), C.byref(m), C.byref(o),
                                   images.data_ptr(), overdraw.data_ptr(), dl.data_ptr() if backward else None,
                                   C.byref(grads) if backward else None, int(reps), int(flush_bytes), C.byref(best),
                                   table, 32, stream)
        if rc < 0:
            _abi.check(rc, self.ctx)
        self.recycle(frame)
        d = default_options(**(options or {}))
        d.update(tile_w=best.tile_w, tile_h=best.tile_h, chunk=best.chunk, schedule=best.schedule)
        rows = [(t.tile_w, t.tile_h, t.chunk, t.schedule, t.ms) for t in table[:rc]]
        del keep
        return d, rows

    def backward(self, frame: Frame, params: dict, dl_dimage: torch.Tensor, out: dict | None = None) -> dict:
        """Path-replay gradients of the frame's render w.r.t. the raw parameters (overwritten into ``out``)."""
        g, keep = _gaussians(params, self.device)
        dl = _check_param(dl_dimage, "dl_dimage", self.device)
        if dl.numel() != frame.n_pixels * 3:
            raise ValueError("dl_dimage must hold 3 values per rendered pixel ([H, W, 3], or packed for a batch)")
        if out is None:
            out = {"d_" + k: torch.empty_like(keep[k]) for k in PARAM_KEYS}
        gr = _abi.Grads(*(out["d_" + k].data_ptr() for k in PARAM_KEYS))
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self.lib.ngs_render_backward(self.ctx, frame.handle, C.byref(g), dl.data_ptr(), C.byref(gr), stream)
        _abi.check(rc, self.ctx)
        return out

    def set_graphs(self, enable: bool):
        """Capture each render phase as a CUDA graph once per configuration and replay it."""
        _abi.check(self.lib.ngs_set_graphs(self.ctx, int(bool(enable))), self.ctx)

    def graph_captures(self) -> int:
        return int(self.lib.ngs_graph_captures(self.ctx))

    def set_timing(self, enable: bool):
        _abi.check(self.lib.ngs_set_timing(self.ctx, int(bool(enable))), self.ctx)

    def stage_times(self) -> dict:
        ms = (C.c_double * _abi.NGS_NUM_STAGES)()
        cnt = (C.c_int64 * _abi.NGS_NUM_STAGES)()
        self.lib.ngs_stage_times(self.ctx, ms, cnt, _abi.NGS_NUM_STAGES)
        return {name: (ms[i], cnt[i]) for i, name in enumerate(_abi.STAGES)}

    def reset_stage_times(self):
        self.lib.ngs_reset_stage_times(self.ctx)

    def launch_count(self) -> int:
        return int(self.lib.ngs_launch_count(self.ctx))

    def set_checked(self, enable: bool):
        """Checked mode: renders refuse NaN / infinite parameters (NGSError naming the array)."""
        _abi.check(self.lib.ngs_set_checked(self.ctx, int(bool(enable))), self.ctx)

    def memory_usage(self, frame: Frame | None = None) -> tuple:
        """(context bytes, frame bytes) of device memory held now."""
        a, b = C.c_size_t(), C.c_size_t()
        self.lib.ngs_memory_usage(self.ctx, frame.handle if frame is not None else None, C.byref(a), C.byref(b))
        return int(a.value), int(b.value)

    def measure_peak(self, kind: int, seconds: float = 1.0) -> float:
        """Measured throughput of a pipe (_abi.NGS_PEAK_*): FLOP/s or ex2 results per second."""
        rate = C.c_double()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _abi.check(self.lib.ngs_measure_peak(self.ctx, int(kind), float(seconds), C.byref(rate), stream), self.ctx)
        return float(rate.value)


def workspace_bytes(n: int, cameras, options=None, n_pairs: int = 0) -> dict:
    """Device bytes a render of n Gaussians from ``cameras`` (one dict or a list) and its backward allocate in
    a fresh context and frame, with the pair buffers sized for ``n_pairs`` (ngs_workspace_bytes). No
    device call."""
    cams = [cameras] if isinstance(cameras, dict) else list(cameras)
    arr = (_abi.Camera * len(cams))(*(_camera(c) for c in cams))
    out = _abi.Workspace()
    rc = _abi.load().ngs_workspace_bytes(int(n), arr, len(cams), C.byref(_options(options)), int(n_pairs), C.byref(out))
    if rc != _abi.NGS_OK:
        raise _abi.NGSError(f"ngs_workspace_bytes: invalid arguments (status {rc})", rc)
    return {k: int(getattr(out, k)) for k, _ in _abi.Workspace._fields_}


_renderers = threading.local()


def default_renderer(device=None) -> Renderer:
    dev = torch.device("cuda") if device is None else torch.device(device)
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    cache = getattr(_renderers, "by_device", None)
    if cache is None:
        cache = _renderers.by_device = {}
    if dev not in cache:
        cache[dev] = Renderer(dev)
    return cache[dev]


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, camera, model, options, renderer, means, log_scales, quats, opacity_logits, sh):
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)
        image, overdraw, frame = renderer.render(params, camera, model, options)
        ctx.frame, ctx.renderer = frame, renderer
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh)
        ctx.mark_non_differentiable(overdraw)
        return image, overdraw

    @staticmethod
    def backward(ctx, dl_dimage, _dl_overdraw):
        means, log_scales, quats, opacity_logits, sh = ctx.saved_tensors
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)
        grads = ctx.renderer.backward(ctx.frame, params, dl_dimage.contiguous())
        ctx.renderer.recycle(ctx.frame)
        ctx.frame = None
        return (None, None, None, None, *(grads["d_" + k] for k in PARAM_KEYS))


def render(params: dict, camera: dict, model="sup", options=None, renderer: Renderer | None = None):
    """Differentiable render: returns (image [H,W,3], overdraw [H,W]); gradients reach the five parameter
    tensors of ``params`` through the library's path-replay backward."""
    renderer = renderer or default_renderer(params["means"].device)
    return _RenderFn.apply(camera, model, options, renderer, *(params[k] for k in PARAM_KEYS))
