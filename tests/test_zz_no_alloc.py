"""ngs_render_backward_static: the backward for callers that cannot let the library allocate device
memory (a fixed memory budget owned by the application, or a loop where cudaMalloc's implicit device
synchronisation is not acceptable). Called through the C ABI and checked against ngs_render_backward on
two calls in a row (the static scratch is shared and must be cleared by each call). Collected last so
that a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer, _gaussians  # noqa: E402
from tests.gpu_util import describe_mismatch, grad_mismatch  # noqa: E402


def _static_backward(r, frame, params, dl):
    g, keep = _gaussians(params, r.device)
    out = {"d_" + k: torch.full_like(keep[k], float("nan")) for k in PARAM_KEYS}
    gr = _abi.Grads(*(out["d_" + k].data_ptr() for k in PARAM_KEYS))
    rc = _abi.load().ngs_render_backward_static(r.ctx, frame.handle, C.byref(g), dl.data_ptr(), C.byref(gr),
                                                torch.cuda.current_stream(r.device).cuda_stream)
    return rc, out


def test_static_backward_matches_backward_twice():
    r = Renderer("cuda:0")
    scene, cam = synth.clustered_scene(20000, seed=8, sh_degree=3), synth.outside_camera(320, 240)
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda() for k in PARAM_KEYS}
    g = synth.upstream_gradient(240, 320, seed=5)
    dl = torch.from_numpy(g).cuda()
    for model in ("exp", "sub", "lin", "sup"):
        _, _, frame = r.render(params, cam, model)
        ref = r.backward(frame, params, dl)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        # the same criterion as the oracle parity tests; the two calls run the same kernels and differ only
        # in the order of their float atomics, which the oracle's per-gradient error scale bounds
        scales = oracle.render(scene, cam, model, nthreads=8, dl_dimage=g)
        for _ in range(2):
            rc, out = _static_backward(r, frame, params, dl)
            assert rc == _abi.NGS_OK, _abi.load().ngs_last_error(r.ctx)
            torch.cuda.synchronize()
            for k in PARAM_KEYS:
                a = out["d_" + k].cpu().numpy()
                bad = grad_mismatch(a, ref["d_" + k], scale=scales["s_" + k])
                assert not bad.any(), (model, k, describe_mismatch(a, ref["d_" + k], bad, scales["s_" + k]))
        r.recycle(frame)
    r.close()


def test_static_backward_rejects_frames_beyond_its_limit():
    r = Renderer("cuda:0")
    scene = synth.tiny_scene(0, n=262145)
    cam = synth.pinhole(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 32, 32, 40.0, 40.0)
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda() for k in PARAM_KEYS}
    _, _, frame = r.render(params, cam, "sup")
    rc, _ = _static_backward(r, frame, params, torch.zeros((32, 32, 3), device="cuda"))
    assert rc == _abi.NGS_ERR_INVALID_ARG
    assert b"262144" in _abi.load().ngs_last_error(r.ctx)
    r.close()
