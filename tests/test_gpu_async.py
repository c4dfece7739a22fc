"""Asynchronous renders (ngs_frame_set_async / ngs_frame_status): the whole pipeline enqueued without the
host synchronisation after binning, sized by the frame's pair capacity.

* a render that fits its capacity is bit-identical to the synchronous render (image, overdraw, replay
  state through the backward), with and without CUDA graphs, single view and batch;
* a render whose pairs exceed the capacity writes only the pairs that fit, is reported by
  ngs_frame_status as NGS_ERR_CAPACITY, grows the capacity, and the next render succeeds and is exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Frame, Renderer  # noqa: E402
from tests.gpu_util import upload  # noqa: E402


@pytest.fixture(scope="module")
def rnd():
    r = Renderer("cuda:0")
    yield r
    r.close()


def _render_backward(rnd, frame, params, cam, model, dl, opts=None):
    img, od, frame = rnd.render(params, cam, model, opts, frame=frame)
    grads = rnd.backward(frame, params, dl)
    torch.cuda.synchronize()
    return img.cpu().numpy(), od.cpu().numpy(), {k: v.cpu().numpy() for k, v in grads.items()}


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("model", ["exp", "sup"])
def test_async_render_matches_sync(rnd, model, graphs):
    scene, cam = synth.clustered_scene(20000, seed=21, sh_degree=3), synth.outside_camera(250, 170, 13.0)
    params = upload(scene)
    dl = torch.from_numpy(synth.upstream_gradient(cam["height"], cam["width"], seed=5)).cuda()
    rnd.set_graphs(graphs)
    try:
        ref_frame = rnd.frame()
        ref_img, ref_od, ref_g = _render_backward(rnd, ref_frame, params, cam, model, dl)
        ref_pairs = ref_frame.view()["n_pairs"]
        f = Frame(rnd)  # a new frame: no capacity yet
        f.set_async(True)
        _render_backward(rnd, f, params, cam, model, dl)  # no capacity yet: synchronous, sets one
        assert f.status() == ref_pairs
        for _ in range(3):  # asynchronous from here on
            img, od, g = _render_backward(rnd, f, params, cam, model, dl)
            assert np.array_equal(img, ref_img) and np.array_equal(od, ref_od)
            for k in PARAM_KEYS:  # float atomics: equal up to the order of additions
                a, b = g["d_" + k], ref_g["d_" + k]
                assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max()), k
            assert f.status() == ref_pairs
        f.release()
        rnd.recycle(ref_frame)
    finally:
        rnd.set_graphs(False)


@pytest.mark.parametrize("graphs", [False, True])
def test_async_capacity_exceeded_then_exact(rnd, graphs):
    small = upload(synth.tiny_scene(3))
    big_scene = synth.clustered_scene(30000, seed=22, sh_degree=3)
    big = upload(big_scene)
    cam = synth.outside_camera(240, 160, 12.0)
    rnd.set_graphs(graphs)
    try:
        ref_img, ref_od, ref_f = rnd.render(big, cam, "lin")
        ref_img, ref_od = ref_img.cpu().numpy(), ref_od.cpu().numpy()
        ref_pairs = ref_f.view()["n_pairs"]
        f = Frame(rnd)
        f.set_async(True)
        rnd.render(small, cam, "lin", frame=f)  # synchronous: a capacity sized for the small scene
        small_pairs = f.status()
        assert ref_pairs > small_pairs + small_pairs // 4 + 1024  # the big scene cannot fit
        rnd.render(big, cam, "lin", frame=f)  # asynchronous, over capacity: writes what fits
        with pytest.raises(_abi.CapacityExceeded):
            f.status()
        img, od, _ = rnd.render(big, cam, "lin", frame=f)  # the capacity has grown
        assert f.status() == ref_pairs
        assert np.array_equal(img.cpu().numpy(), ref_img) and np.array_equal(od.cpu().numpy(), ref_od)
        f.release()
        rnd.recycle(ref_f)
    finally:
        rnd.set_graphs(False)


def test_async_batch_matches_sync(rnd):
    scene = synth.clustered_scene(15000, seed=23, sh_degree=2)
    params = upload(scene)
    cams = [synth.outside_camera(200, 120, 12.0), synth.outside_camera(96, 160, 14.0),
            synth.outside_camera(150, 150, 11.0)]
    ref_img, ref_od, ref_f = rnd.render_batch(params, cams, "sub")
    ref_img, ref_od = ref_img.cpu().numpy(), ref_od.cpu().numpy()
    f = Frame(rnd)
    f.set_async(True)
    rnd.render_batch(params, cams, "sub", frame=f)
    f.status()
    img, od, _ = rnd.render_batch(params, cams, "sub", frame=f)
    assert f.status() == ref_f.view()["n_pairs"]
    assert np.array_equal(img.cpu().numpy(), ref_img) and np.array_equal(od.cpu().numpy(), ref_od)
    f.release()
    rnd.recycle(ref_f)


def test_status_without_render_is_an_error(rnd):
    f = Frame(rnd)
    with pytest.raises(_abi.NGSError):
        f.status()
    f.set_async(True)
    with pytest.raises(_abi.NGSError):
        f.status()
    f.release()
