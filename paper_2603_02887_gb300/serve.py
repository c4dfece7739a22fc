"""Serving over the library's native render server (``ngs_server_*``): resident scenes, continuous
batching, admission by sort-buffer memory, latency accounting.

``Server`` marshals arguments only; batching, admission and the render itself run in the library (its
worker threads and CUDA kernels). ``run_poisson`` drives a server with a seeded Poisson arrival process;
``run_one_at_a_time`` serves the same arrivals with one render call at a time, for comparison.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np
import torch

from . import _abi
from .render import _camera, _gaussians, _options, model_spec


class Server:
    def __init__(self, workers: int = 4, max_batch_views: int = 16, mem_budget: int = 8 << 30, graphs: bool = False,
                 options=None, device=None):
        self.lib = _abi.load()
        self.device = torch.device("cuda") if device is None else torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        cfg = _abi.ServerConfig()
        self.lib.ngs_default_server_config(C.byref(cfg))
        cfg.workers, cfg.max_batch_views, cfg.mem_budget = int(workers), int(max_batch_views), int(mem_budget)
        cfg.graphs = int(bool(graphs))
        cfg.options = _options(options)
        self.handle = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.ngs_server_create(C.byref(cfg), C.byref(self.handle))
        if rc != _abi.NGS_OK:
            raise _abi.NGSError(f"ngs_server_create failed ({rc})")
        self._scenes = []    # parameter tensors kept alive while the server may read them
        self._inflight = {}  # tag -> (image, overdraw) until completion
        self._next_tag = 0

    def add_scene(self, params: dict) -> int:
        g, keep = _gaussians(params, self.device)
        sid = C.c_int32()
        self._check(self.lib.ngs_server_add_scene(self.handle, C.byref(g), C.byref(sid)))
        self._scenes.append(keep)
        return sid.value

    def submit(self, scene: int, camera: dict, model="sup", image: torch.Tensor | None = None,
               overdraw: torch.Tensor | None = None, tag: int | None = None) -> int:
        cam = _camera(camera)
        if image is None:
            image = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=self.device)
        if overdraw is None:
            overdraw = torch.empty((cam.height, cam.width), dtype=torch.int32, device=self.device)
        if image.numel() != cam.height * cam.width * 3 or overdraw.numel() != cam.height * cam.width:
            raise ValueError("output buffers do not match the camera size")
        if tag is None:
            tag = self._next_tag
            self._next_tag += 1
        kind, param = model_spec(model)
        req = _abi.Request(int(scene), _abi.Model(kind, param), cam, image.data_ptr(), overdraw.data_ptr(), int(tag))
        self._inflight[int(tag)] = (image, overdraw)  # before the workers can complete it
        rc = self.lib.ngs_server_submit(self.handle, C.byref(req))
        if rc != _abi.NGS_OK:
            self._inflight.pop(int(tag), None)
            raise _abi.NGSError(f"request refused ({rc}): scene id, camera or model out of range")
        return int(tag)

    def poll(self, wait_ms: int = 0, cap: int = 256) -> list:
        """Completed requests: dicts with tag, status, batch_views, submit_s/start_s/done_s (server clock),
        pairs, image, overdraw."""
        buf = (_abi.Completion * cap)()
        n = self.lib.ngs_server_poll(self.handle, buf, cap, int(wait_ms))
        if n < 0:
            self._check(n)
        out = []
        for c in buf[:n]:
            img, od = self._inflight.pop(c.tag, (None, None))
            out.append(dict(tag=c.tag, status=c.status, batch_views=c.batch_views, submit_s=c.submit_s,
                            start_s=c.start_s, done_s=c.done_s, pairs=c.pairs, image=img, overdraw=od))
        return out

    def stats(self) -> dict:
        s = _abi.ServerStats()
        self._check(self.lib.ngs_server_get_stats(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in _abi.ServerStats._fields_}

    def last_error(self) -> str:
        m = self.lib.ngs_server_last_error(self.handle)
        return m.decode() if m else ""

    def close(self):
        if self.handle:
            self.lib.ngs_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != _abi.NGS_OK:
            raise _abi.NGSError(f"ngs server error {rc}: {self.last_error()}")


def poisson_arrivals(n: int, rate: float, seed: int = 3) -> np.ndarray:
    """Arrival times (seconds from 0) of n requests of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def _latency_summary(lat_ms, elapsed_s, n):
    lat = np.asarray(lat_ms)
    return {"requests": int(n), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "max_ms": round(float(lat.max()), 3), "frames_per_s": round(n / elapsed_s, 2),
            "elapsed_s": round(elapsed_s, 3)}


def run_poisson(server: Server, requests: list, arrivals: np.ndarray, outputs: list | None = None) -> dict:
    """Submit requests[i] = (scene, camera, model) at arrivals[i] (seconds after the start) and collect every
    completion. Latency = completion - arrival. outputs: optional per-request (image, overdraw) buffers."""
    n = len(requests)
    t0 = time.perf_counter()
    base = server.stats()["now_s"]
    i = 0
    done = {}
    while len(done) < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            sc, cam, model = requests[i]
            img, od = outputs[i] if outputs else (None, None)
            server.submit(sc, cam, model, image=img, overdraw=od, tag=i)
            i += 1
        wait = 0 if i < n and arrivals[i] - (time.perf_counter() - t0) < 1e-3 else 1
        for c in server.poll(wait_ms=wait):
            done[c["tag"]] = c
    elapsed = time.perf_counter() - t0
    bad = [c for c in done.values() if c["status"] != 0]
    if bad:
        raise _abi.NGSError(f"{len(bad)} requests failed: {server.last_error()}")
    lat = [(done[k]["done_s"] - base - arrivals[k]) * 1e3 for k in range(n)]
    out = _latency_summary(lat, elapsed, n)
    sizes = np.array([c["batch_views"] for c in done.values()])
    out["mean_batch_views"] = round(float(sizes.mean()), 3)
    out["results"] = done
    return out


def run_one_at_a_time(renderer, scenes: list, requests: list, arrivals: np.ndarray, options=None,
                      outputs: list | None = None) -> dict:
    """The same arrivals served by one render call at a time on one stream (no batching, no overlap):
    each request starts at max(its arrival, the previous completion)."""
    n = len(requests)
    frames = {}
    lat = []
    t0 = time.perf_counter()
    for i, (sc, cam, model) in enumerate(requests):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        key = (sc, cam["width"], cam["height"])
        img, od = outputs[i] if outputs else (None, None)
        _, _, frames[key] = renderer.render(scenes[sc], cam, model, options, frame=frames.get(key), image=img,
                                            overdraw=od)
        torch.cuda.current_stream().synchronize()
        lat.append((time.perf_counter() - t0 - arrivals[i]) * 1e3)
    elapsed = time.perf_counter() - t0
    for f in frames.values():
        renderer.recycle(f)
    return _latency_summary(lat, elapsed, n)
