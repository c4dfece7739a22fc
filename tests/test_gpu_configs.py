"""GPU parity at the full sizes of the benchmark configurations, in the launch configuration bench.py
times (its per-model launch options, bench.TUNED_OPTIONS: exponential on 8x8 tiles, the quadratic models
on 16x16), on outputs the FP64 oracle computes one by one: windows of the full frame.

* single large view: 500k clustered Gaussians (SH 3) at 1920x1080, forward for the four models, on three
  windows (centre, an off-centre region, and a stretch of the bottom edge, where the 16-pixel tiles are
  ragged since 1080 = 67.5 x 16);
* the pair sort of the exponential model's 8x8 tiles at 1920x1080 with 500k and 2M Gaussians: properties
  of the whole sorted array, and sampled tiles against the oracle's list for each;
* batched multi-view: 3M clustered Gaussians from 32 cameras of uneven size in one batch, forward for the
  four models on windows of three views, and the batch's gradient from an upstream gradient on one
  view's window against the oracle's gradients of that window;
* differentiation: 1M clustered Gaussians at 1297x840, forward + path-replay backward for the four models
  with an L1-type upstream gradient restricted to a 256x256 window, against the oracle's gradients of that
  window; and the GPU's gradient on 64 random raw parameters against central differences of the FP64
  oracle.
Every pixel of a window is checked against the oracle's outcomes for it (tests/parity.py).
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
from oracle import binning  # noqa: E402
from paper_2603_02887_gb300 import synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer  # noqa: E402
from tests import parity  # noqa: E402
from tests.gpu_util import frame_arrays, upload  # noqa: E402

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
        ref = oracle.render(scene, cam, model, window=win, nthreads=NT, outcomes=True)
        m = parity.assert_forward(img[y0:y0 + h, x0:x0 + w], od[y0:y0 + h, x0:x0 + w], ref, label=f"{model} {win}")
        assert m.n_unresolved == 0, m.summary()
        print(f"[parity] 500k/1080p {model} window {win}: {m.summary()}")
        assert ref["overdraw"].mean() > 0.5, win  # the windows are not empty


@pytest.mark.parametrize("n", [500_000, 2_000_000])
def test_pair_sort_full_size(rnd, n):
    """The pair sort at full size in the exponential model's bench launch options (8x8 tiles, 1920x1080):
    500k Gaussians give about 4.2M pairs (the sort's tiles of 1024 keys), 2M more than 2^23 (tiles of 4096
    keys). Over the whole array: tiles non-decreasing, each tile's pairs in (depth, index) order, the ranges
    the runs of each tile. Tile by tile against the oracle's list (oracle/binning.tile_lists on the GPU's own
    records): the 8 longest lists and 56 random non-empty ones."""
    scene = synth.clustered_scene(n, seed=0 if n == 500_000 else 4, sh_degree=3)
    cam = synth.outside_camera(1920, 1080)
    _, _, frame = rnd.render(upload(scene), cam, "exp", OPTS["exp"])
    fa = frame_arrays(frame)
    keys, vals, ranges = fa["keys"], fa["values"], fa["ranges"].astype(np.int64)
    P = len(keys)
    assert P > (1 << 23) if n > 500_000 else P > 4_000_000, P
    tile, z = (keys >> np.uint64(32)).astype(np.int64), (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.all(np.diff(tile) >= 0)
    same = tile[1:] == tile[:-1]
    dz = np.diff(z)
    assert np.all(dz[same] >= 0)
    tie = same & (dz == 0)
    assert np.all(vals[1:][tie] > vals[:-1][tie])
    lens = ranges[:, 1] - ranges[:, 0]
    assert lens.sum() == P
    nz = np.nonzero(lens)[0]
    assert np.array_equal(tile[ranges[nz, 0]], nz) and np.array_equal(tile[ranges[nz, 1] - 1], nz)
    rng = np.random.default_rng(n)
    pick = sorted(set(np.argsort(lens)[-8:].tolist()) | set(rng.choice(nz, 56, replace=False).tolist()))
    exp = binning.tile_lists(fa["records"], fa["view"]["log2_alpha_min"], 8, 8, 1920, 1080, pick)
    for t in pick:
        s, e = ranges[t]
        assert np.array_equal(vals[s:e], exp[t]), t
    print(f"[parity] pair sort {n} Gaussians, 1920x1080 8x8: {P} pairs; {len(pick)} tiles checked, longest "
          f"{int(lens.max())}")
    rnd.recycle(frame)


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
    g = synth.upstream_gradient(h, w, seed=11)
    ref = oracle.render(scene, cam, model, window=win, nthreads=NT, dl_dimage=g.astype(np.float64), outcomes=True)
    m = parity.assert_forward(image.cpu().numpy()[y0:y0 + h, x0:x0 + w], overdraw.cpu().numpy()[y0:y0 + h, x0:x0 + w],
                              ref, label=model)
    assert m.n_unresolved == 0, m.summary()
    dl = np.zeros((cam["height"], cam["width"], 3), np.float32)
    dl[y0:y0 + h, x0:x0 + w] = g
    grads = rnd.backward(frame, params, torch.from_numpy(dl).cuda())
    torch.cuda.synchronize()
    rep = parity.assert_gradients({k: v.cpu().numpy() for k, v in grads.items()}, ref, m, label=model)
    print(f"[parity] 1M/1297x840 crop {model}: {m.summary()}; {rep.summary()}")
    assert np.count_nonzero(ref["d_opacity_logits"]) > 1000  # the window reaches many Gaussians


def _window_subscene(scene, cam, win):
    """The Gaussians that can reach a window: their candidate disc (alpha >= alpha_min 2^-0.5, the
    oracle's widest candidate threshold) around the projected mean meets the window, with a 2 px margin.
    A render of the window from them equals the full scene's."""
    p = oracle.project(scene, cam)
    rec = p["rec"]
    A, B, C, aleph = rec[:, 2], rec[:, 3], rec[:, 4], rec[:, 5]
    lam_min = 0.5 * (A + C) - np.sqrt(0.25 * (A - C) ** 2 + B ** 2)  # smallest eigenvalue of the conic
    thr = np.float32(1 / 255.0) * 2 ** -0.5
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.sqrt(np.maximum(2 * np.log(aleph / thr), 0) / lam_min) + 2
    x0, y0, w, h = win
    sel = (p["z32"] > np.float32(0.2)) & (aleph >= thr) & (lam_min > 0)
    sel &= (rec[:, 0] + r >= x0) & (rec[:, 0] - r <= x0 + w) & (rec[:, 1] + r >= y0) & (rec[:, 1] - r <= y0 + h)
    idx = np.nonzero(sel)[0]
    return {k: v[idx] for k, v in scene.items()}, idx


@pytest.fixture(scope="module")
def fd_window(diff_scene):
    scene, cam = diff_scene
    win = (584, 364, 128, 128)
    sub, idx = _window_subscene(scene, cam, win)
    return win, sub, idx


@pytest.mark.parametrize("model", MODELS)
def test_differentiation_1m_finite_differences(rnd, diff_scene, fd_window, model):
    """The GPU's path-replay gradient on 64 random raw parameters against central differences of the
    FP64 oracle (L = sum(g * image) over a 128x128 window of the 1M-Gaussian frame, g nonzero only there),
    at relative 1e-3, for each of the four models.

    The oracle renders the window from the Gaussians that can reach it (the same image as from the whole
    scene, checked). Steps are h = 1e-5 max(1, |theta|); a sample is redrawn when any pixel's composited
    list, stop or clamp state differs between the two sides of the stencil (L is not differentiable
    there). Where a pixel's GPU result took another legitimate outcome than the FP64 walk, the expected
    value carries that outcome's difference (tests/parity.py); the tolerance is that of the crop test."""
    scene, cam = diff_scene
    win, sub, idx = fd_window
    x0, y0, w, h = win
    params = upload(scene)
    img0, od0, frame = rnd.render(params, cam, model, OPTS[model])
    gw = synth.upstream_gradient(h, w, seed=12).astype(np.float64)
    g = np.zeros((cam["height"], cam["width"], 3), np.float32)
    g[y0:y0 + h, x0:x0 + w] = gw
    grads = {k: v.cpu().numpy() for k, v in rnd.backward(frame, params, torch.from_numpy(g).cuda()).items()}
    ref = oracle.render(sub, cam, model, window=win, nthreads=NT, dl_dimage=gw, outcomes=True)
    if model == "sup":  # the window's Gaussians render the same image as the whole scene
        full = oracle.render(scene, cam, model, window=win, nthreads=NT)
        assert np.array_equal(ref["image"], full["image"]) and np.array_equal(ref["overdraw"], full["overdraw"])
    m = parity.assert_forward(img0.cpu().numpy()[y0:y0 + h, x0:x0 + w], od0.cpu().numpy()[y0:y0 + h, x0:x0 + w], ref)
    gref = parity.reference_gradients(ref, m)
    live = np.nonzero(np.abs(ref["d_opacity_logits"]) > 0.05 * np.abs(ref["d_opacity_logits"]).max())[0]
    rng = np.random.default_rng(13)
    checked, worst = 0, 0.0
    for _ in range(400):
        if checked == 64:
            break
        key = PARAM_KEYS[rng.integers(0, len(PARAM_KEYS))]
        li = int(rng.choice(live))
        flat = sub[key].reshape(len(sub[key]), -1)
        j = int(rng.integers(0, flat.shape[1]))
        exp_adj = gref.d[key][li, j] - ref["d_" + key].reshape(len(sub[key]), -1)[li, j]
        th = float(flat[li, j])
        hstep = 1e-5 * max(1.0, abs(th))
        outs = []
        for sgn in (1, -1):
            s2 = {k: v.astype(np.float64).copy() for k, v in sub.items()}
            s2[key].reshape(len(s2[key]), -1)[li, j] = th + sgn * hstep
            outs.append(oracle.render(s2, cam, model, window=win, nthreads=NT))
        if not all(np.array_equal(o["signature"], ref["signature"]) for o in outs):
            continue
        fd = (np.sum(gw * outs[0]["image"]) - np.sum(gw * outs[1]["image"])) / (2 * hstep)
        expected = fd + exp_adj
        an = float(grads["d_" + key].reshape(len(scene[key]), -1)[idx[li], j])
        floor = parity.FLOOR_REL * np.abs(gref.d[key]).max()
        tol = (parity.GRAD_REL * max(abs(expected), floor) + gref.allow[key][li, j]
               + parity.SCALE_REL * gref.s[key][li, j])
        assert abs(an - expected) <= tol, (key, li, j, an, expected, fd, tol)
        worst = max(worst, abs(an - expected) / max(abs(expected), floor))
        checked += 1
    assert checked == 64
    print(f"[parity] 1M/1297x840 {model}: finite differences of the FP64 oracle, 64 samples, worst "
          f"|an - fd| / max(|fd|, floor) = {worst:.2e}")


# The batched workload's launch options: what ngs_autotune picks for it on GB300 (bench.py's batched leg
# tunes them on every run; they do not change any result).
BATCH_OPTS = {"exp": dict(tile_w=16, tile_h=16, chunk=128, schedule="tiles"),
              **{m: dict(tile_w=16, tile_h=32, chunk=256, schedule="tiles") for m in ("sub", "lin", "sup")}}


@pytest.fixture(scope="module")
def batched_scene():
    return synth.clustered_scene(3_000_000, seed=0, sh_degree=3), synth.orbit_cameras(32, radius=12.0, seed=2)


@pytest.mark.parametrize("model", MODELS)
def test_batched_3m_32_views(rnd, batched_scene, model):
    """The batched configuration at full size (3M Gaussians, 32 views of 640x360 .. 1920x1080 in one
    batch): every pixel of a 40x40 window at the centre of views 0, 13 and 31 against the oracle's outcomes;
    then the batch's gradient for an upstream gradient that is nonzero on a 48x48 window of view 13 only,
    against the oracle's gradients of that window (rendered from the Gaussians that can reach it: every
    other Gaussian's GPU gradient must be exactly zero)."""
    scene, cams = batched_scene
    params = upload(scene)
    images, overdraw, frame = rnd.render_batch(params, cams, model, options=BATCH_OPTS[model])
    imgs, ods = frame.split(images), frame.split(overdraw)
    for v in (0, 13, 31):
        c = cams[v]
        win = (c["width"] // 2 - 20, c["height"] // 2 - 20, 40, 40)
        x0, y0, w, h = win
        ref = oracle.render(scene, c, model, window=win, nthreads=NT, outcomes=True)
        m = parity.assert_forward(imgs[v].cpu().numpy()[y0:y0 + h, x0:x0 + w],
                                  ods[v].cpu().numpy()[y0:y0 + h, x0:x0 + w], ref, label=f"{model} view {v}")
        assert m.n_unresolved == 0, m.summary()
        assert ref["overdraw"].mean() > 0.5, (v, win)
        print(f"[parity] batched 3M x 32 {model} view {v} {win}: {m.summary()}")
    v = 13
    c = cams[v]
    win = (c["width"] // 2 + 16, c["height"] // 2 - 24, 48, 48)
    x0, y0, w, h = win
    gw = synth.upstream_gradient(h, w, seed=21)
    base = int(frame.view()["view_pixel_base"][v])
    dl = torch.zeros((images.shape[0], 3), dtype=torch.float32)
    rows = base + (np.arange(y0, y0 + h)[:, None] * c["width"] + np.arange(x0, x0 + w)[None, :]).reshape(-1)
    dl[torch.from_numpy(rows)] = torch.from_numpy(gw.reshape(-1, 3))
    grads = {k: t.cpu().numpy() for k, t in rnd.backward(frame, params, dl.cuda()).items()}
    sub, idx = _window_subscene(scene, c, win)
    ref = oracle.render(sub, c, model, window=win, nthreads=NT, dl_dimage=gw.astype(np.float64), outcomes=True)
    m = parity.assert_forward(imgs[v].cpu().numpy()[y0:y0 + h, x0:x0 + w], ods[v].cpu().numpy()[y0:y0 + h, x0:x0 + w],
                              ref, label=f"{model} view {v} gradient window")
    others = np.ones(len(scene["means"]), bool)
    others[idx] = False
    for k in PARAM_KEYS:
        assert not np.any(grads["d_" + k][others]), (model, k)  # Gaussians that cannot reach the window
    rep = parity.assert_gradients({k: g[idx] for k, g in grads.items()}, ref, m, label=model)
    assert np.count_nonzero(ref["d_opacity_logits"]) > 100
    print(f"[parity] batched 3M x 32 {model} view {v} gradients {win}: {m.summary()}; {rep.summary()}")
    rnd.recycle(frame)

