"""On the GPU: ngs_workspace_bytes against a render's actual device allocations, checked mode, and the
peak microbenchmarks' sanity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import Renderer, default_options, workspace_bytes  # noqa: E402
from tests.gpu_util import upload  # noqa: E402


@pytest.mark.parametrize("schedule", ["tiles", "persistent"])
def test_workspace_equals_actual_allocation(schedule):
    scene = synth.clustered_scene(20000, seed=4, sh_degree=3)
    cams = [synth.outside_camera(203, 141, 12.0), synth.outside_camera(320, 180, 13.0)]
    params = upload(scene)
    opts = default_options(schedule=schedule)
    r = Renderer("cuda:0")  # a fresh context and frame: no buffer has grown yet
    img, od, frame = r.render_batch(params, cams, "sup", opts)
    torch.cuda.synchronize()
    pairs = int(frame.view()["n_pairs"])
    ws = workspace_bytes(20000, cams, opts, pairs)
    ctx_b, frame_b = r.memory_usage(frame)
    # frame_view_get composed 64-bit keys into a diagnostics buffer (8 B per pair, rounded)
    keys64 = (max(8 * pairs, 256) + 255) // 256 * 256
    assert frame_b - keys64 == ws["frame_fixed"] + ws["frame_pairs"]
    assert ctx_b == ws["context"]
    g = torch.ones_like(img)
    r.backward(frame, params, g)
    torch.cuda.synchronize()
    ctx_b2, _ = r.memory_usage(frame)
    assert ctx_b2 == ws["context"] + ws["backward"]
    r.close()


def test_checked_mode_refuses_non_finite_parameters():
    scene = synth.tiny_scene(0, n=200)
    cam = synth.tiny_camera()
    r = Renderer("cuda:0")
    good = upload(scene)
    img0, _, _ = r.render(good, cam, "sup")
    r.set_checked(True)
    img1, _, _ = r.render(good, cam, "sup")  # finite parameters: the same image
    assert torch.equal(img0, img1)
    for key, bad in (("means", float("nan")), ("sh", float("inf")), ("opacity_logits", float("-inf"))):
        p = {k: v.clone() for k, v in good.items()}
        p[key].view(-1)[17] = bad
        with pytest.raises(_abi.NGSError, match=key):
            r.render(p, cam, "sup")
        r.set_checked(False)
        r.render(p, cam, "sup")  # the fast path does not scan
        r.set_checked(True)
    r.close()


def test_peak_microbenchmarks_are_plausible():
    r = Renderer("cuda:0")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ffma = r.measure_peak(_abi.NGS_PEAK_FFMA, 0.2)
    ffma2 = r.measure_peak(_abi.NGS_PEAK_FFMA2, 0.2)
    ex2 = r.measure_peak(_abi.NGS_PEAK_EX2, 0.2)
    nominal = sms * 128 * 2 * 2.07e9  # FP32 lanes x 2 FLOP x the maximum SM clock
    assert 0.3 * nominal < ffma < 1.05 * nominal, (ffma, nominal)
    assert 0.3 * nominal < ffma2 < 2.1 * nominal, (ffma2, nominal)
    assert 0.02 * nominal / 2 < ex2 < nominal / 2, (ex2, nominal)
    with pytest.raises(_abi.NGSError):
        r.measure_peak(7, 0.1)
    print(f"[peak] FFMA {ffma / 1e12:.1f} TFLOP/s, FFMA2 {ffma2 / 1e12:.1f} TFLOP/s, ex2 {ex2 / 1e12:.2f} T/s")
    r.close()
