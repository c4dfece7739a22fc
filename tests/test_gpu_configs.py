"""GPU parity at the full sizes of the benchmark configurations, in the launch configuration bench.py
times (its per-model launch options, bench.TUNED_OPTIONS: exponential on 8x8 tiles, the quadratic models
on 16x16), on outputs the FP64 oracle computes one by one: windows of the full frame.

* single large view: 500k clustered Gaussians (SH 3) at 1920x1080, forward for the four models, on three
  windows (centre, an off-centre region, and a stretch of the bottom edge, where the 16-pixel tiles are
  ragged since 1080 = 67.5 x 16);
* differentiation: 1M clustered Gaussians at 1297x840, forward + path-replay backward for the four models
  with an L1-type upstream gradient restricted to a 256x256 window, against the oracle's gradients of that
  window; and central differences of the GPU render itself on 64 random raw parameters.
Inputs are seeded synthetic scenes (paper_2603_02887_gb300.synth); no oracle input comes from the GPU.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2603_02887_gb300 import synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer  # noqa: E402
from tests.gpu_util import describe_mismatch, grad_mismatch, upload  # noqa: E402

MODELS = ["exp", "sub", "lin", "sup"]
NT = os.cpu_count() or 4
OPTS = bench.parse_options()  # the launch options bench.py times


@pytest.fixture(scope="module")
def rnd():
    r = Renderer("cuda:0")
    yield r
    r.close()


@pytest.fixture(scope="module")
def single_view():
    return synth.clustered_scene(500_000, seed=0, sh_degree=3), synth.outside_camera(1920, 1080)


@pytest.mark.parametrize("model", MODELS)
def test_single_view_500k_1080p_windows(rnd, single_view, model):
    scene, cam = single_view
    params = upload(scene)
    image, overdraw, _ = rnd.render(params, cam, model, OPTS[model])
    img, od = image.cpu().numpy(), overdraw.cpu().numpy()
    for win in ((936, 516, 48, 48), (400, 300, 40, 40), (900, 1080 - 13, 64, 13)):
        x0, y0, w, h = win
        ref = oracle.render(scene, cam, model, window=win, nthreads=NT)
        ok = ~ref["fragile"]
        assert ref["fragile"].sum() <= max(2, 0.01 * ok.size)
        err = np.abs(img[y0:y0 + h, x0:x0 + w] - ref["image"])[ok]
        assert err.max() <= 1e-4, (win, err.max())
        assert np.array_equal(od[y0:y0 + h, x0:x0 + w][ok], ref["overdraw"][ok]), win
        assert ref["overdraw"].mean() > 0.5, win  # the windows are not empty


@pytest.fixture(scope="module")
def diff_scene():
    return synth.clustered_scene(1_000_000, seed=0, sh_degree=3), synth.outside_camera(1297, 840)


@pytest.mark.parametrize("model", MODELS)
def test_differentiation_1m_crop_gradients(rnd, diff_scene, model):
    scene, cam = diff_scene
    win = (520, 300, 256, 256)
    x0, y0, w, h = win
    params = upload(scene)
    image, overdraw, frame = rnd.render(params, cam, model, OPTS[model])
    ref0 = oracle.render(scene, cam, model, window=win, nthreads=NT)
    ok = ~ref0["fragile"]
    err = np.abs(image.cpu().numpy()[y0:y0 + h, x0:x0 + w] - ref0["image"])[ok]
    assert err.max() <= 1e-4
    g = synth.upstream_gradient(h, w, seed=11).astype(np.float64) * ok[..., None]
    ref = oracle.render(scene, cam, model, window=win, nthreads=NT, dl_dimage=g)
    dl = np.zeros((cam["height"], cam["width"], 3), np.float32)
    dl[y0:y0 + h, x0:x0 + w] = g
    grads = rnd.backward(frame, params, torch.from_numpy(dl).cuda())
    torch.cuda.synchronize()
    report = {}
    for k in PARAM_KEYS:
        a = grads["d_" + k].cpu().numpy()
        bad = grad_mismatch(a, ref["d_" + k], exclude=ref["fragile_gauss"], scale=ref["s_" + k])
        if bad.any():
            report[k] = f"{int(bad.sum())} of {bad.size}: " + describe_mismatch(a, ref["d_" + k], bad, ref["s_" + k])
    assert not report, report
    assert np.count_nonzero(ref["d_opacity_logits"]) > 1000  # the window reaches many Gaussians


def test_differentiation_1m_finite_differences(rnd, diff_scene):
    """Central differences of the GPU render (loss accumulated in FP64) on 64 random raw parameters of
    Gaussians that reach the window, against the GPU's path-replay gradient. A sample whose overdraw map
    changes between the two sides of the stencil is redrawn (a decision flipped)."""
    scene, cam = diff_scene
    win = (520, 300, 256, 256)
    x0, y0, w, h = win
    model = "sup"
    params = upload(scene)
    _, od0, frame = rnd.render(params, cam, model, OPTS[model])
    g = np.zeros((cam["height"], cam["width"], 3), np.float32)
    g[y0:y0 + h, x0:x0 + w] = synth.upstream_gradient(h, w, seed=12)
    gt = torch.from_numpy(g).cuda()
    grads = {k: v.cpu().numpy() for k, v in rnd.backward(frame, params, gt).items()}
    live = np.nonzero(np.abs(grads["d_opacity_logits"]) > 0.05 * np.abs(grads["d_opacity_logits"]).max())[0]
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(400):
        if checked == 64:
            break
        key = PARAM_KEYS[rng.integers(0, len(PARAM_KEYS))]
        gi = int(rng.choice(live))
        flat = params[key].view(params[key].shape[0], -1)
        j = int(rng.integers(0, flat.shape[1]))
        an = grads["d_" + key].reshape(len(scene[key]), -1)[gi, j]
        if abs(an) < 1e-2 * np.abs(grads["d_" + key]).max():
            continue
        th = float(flat[gi, j])
        hstep = 3e-4 * max(1.0, abs(th))
        losses, ods = [], []
        for sgn in (1, -1):
            flat[gi, j] = th + sgn * hstep
            img, od, _ = rnd.render(params, cam, model, OPTS[model])
            losses.append(float((img.double() * gt.double()).sum()))
            ods.append(od)
        flat[gi, j] = th
        if not (torch.equal(ods[0], od0) and torch.equal(ods[1], od0)):
            continue
        fd = (losses[0] - losses[1]) / (2 * hstep)
        assert abs(fd - an) <= 0.05 * abs(an) + 1e-3, (key, gi, j, fd, an)
        checked += 1
    assert checked == 64
