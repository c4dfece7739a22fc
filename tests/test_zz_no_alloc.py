"""ngs_render_backward_static: the backward for callers that cannot let the library allocate device
memory (an application that owns a fixed device-memory budget, or a loop where cudaMalloc's implicit
device synchronisation is not acceptable).

Called through the C ABI on two calls in a row (the static scratch is shared and each call must clear
it): its gradients are held to the FP64 oracle (every pixel and Gaussian, tests/parity.py) and to
ngs_render_backward, up to the order of the float additions. A second test shows that a call allocates
no device memory, where ngs_render_backward on a fresh context does. Collected last, so that a run that
stops at the first failure has already run every other test."""
import ctypes as C
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer, _gaussians  # noqa: E402
from tests import parity  # noqa: E402

NT = os.cpu_count() or 4


def _call(r, fn, frame, params, dl, out):
    """One backward through the C ABI into the preallocated ``out`` (no torch allocation here)."""
    g, _ = _gaussians(params, r.device)
    gr = _abi.Grads(*(out["d_" + k].data_ptr() for k in PARAM_KEYS))
    return fn(r.ctx, frame.handle, C.byref(g), dl.data_ptr(), C.byref(gr),
              torch.cuda.current_stream(r.device).cuda_stream)


def _outputs(params):
    return {"d_" + k: torch.full_like(params[k], float("nan")) for k in PARAM_KEYS}


def test_static_backward_matches_oracle_and_backward_twice():
    lib = _abi.load()
    r = Renderer("cuda:0")
    scene, cam = synth.clustered_scene(20000, seed=8, sh_degree=3), synth.outside_camera(320, 240)
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda() for k in PARAM_KEYS}
    g = synth.upstream_gradient(240, 320, seed=5)
    dl = torch.from_numpy(g).cuda()
    for model in ("exp", "sub", "lin", "sup"):
        image, overdraw, frame = r.render(params, cam, model)
        ref = oracle.render(scene, cam, model, nthreads=NT, dl_dimage=g.astype(np.float64), outcomes=True)
        m = parity.assert_forward(image.cpu().numpy(), overdraw.cpu().numpy(), ref, label=model)
        gref = parity.reference_gradients(ref, m)
        out = _outputs(params)
        assert _call(r, lib.ngs_render_backward, frame, params, dl, out) == _abi.NGS_OK
        torch.cuda.synchronize()
        base = {k: out["d_" + k].cpu().numpy() for k in PARAM_KEYS}
        for call in range(2):
            out = _outputs(params)
            rc = _call(r, lib.ngs_render_backward_static, frame, params, dl, out)
            assert rc == _abi.NGS_OK, lib.ngs_last_error(r.ctx)
            torch.cuda.synchronize()
            got = {k: out["d_" + k].cpu().numpy() for k in PARAM_KEYS}
            rep = parity.compare_gradients(got, gref)
            assert rep.failed == 0 and rep.scaled <= 1e-3 * rep.n, (model, call, rep.summary(), rep.details)
            for k in PARAM_KEYS:
                # the same kernels on the same frame: only the order of the float additions differs, which
                # moves a sum of N terms by at most (N - 1) u sum|terms| (s_* is that sum, N < 1600 here)
                s = ref["s_" + k].reshape(got[k].shape)
                assert np.all(np.abs(got[k] - base[k]) <= 1e-4 * s + 1e-12), (model, call, k)
        r.recycle(frame)
    r.close()


def test_static_backward_allocates_no_device_memory():
    """On a fresh context, after one static call (which looks up the static array and loads the kernels),
    two more static calls leave the device's free memory unchanged; ngs_render_backward on the same frame
    then allocates the context's record-gradient scratch (48 bytes per splat record), which the same
    measurement sees."""
    lib = _abi.load()
    r = Renderer("cuda:0")
    scene, cam = synth.tiny_scene(1, n=200_000), synth.tiny_camera()
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda() for k in PARAM_KEYS}
    dl = torch.from_numpy(synth.upstream_gradient(128, 128, seed=6)).cuda()
    _, _, frame = r.render(params, cam, "sup")
    out = _outputs(params)
    assert _call(r, lib.ngs_render_backward_static, frame, params, dl, out) == _abi.NGS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _call(r, lib.ngs_render_backward_static, frame, params, dl, out) == _abi.NGS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert _call(r, lib.ngs_render_backward, frame, params, dl, out) == _abi.NGS_OK
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free0 - free2 >= 48 * 200_000, (free0, free2)  # the measurement sees an allocation of this size
    r.close()


def test_static_backward_rejects_frames_beyond_its_limit():
    r = Renderer("cuda:0")
    scene = synth.tiny_scene(0, n=262145)
    cam = synth.pinhole(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 32, 32, 40.0, 40.0)
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda() for k in PARAM_KEYS}
    _, _, frame = r.render(params, cam, "sup")
    out = _outputs(params)
    rc = _call(r, _abi.load().ngs_render_backward_static, frame, params, torch.zeros((32, 32, 3), device="cuda"), out)
    assert rc == _abi.NGS_ERR_INVALID_ARG
    assert b"262144" in _abi.load().ngs_last_error(r.ctx)
    r.close()
