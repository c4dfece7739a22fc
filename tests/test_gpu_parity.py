"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: keys, sort order, tile ranges and overdraw are bit-exact; pixels agree to max-abs 1e-4 and
gradients to relative 1e-3 (with a floor of 1e-3 x the tensor's largest gradient), FP32 against FP64.
Every pixel is checked: where a compositing decision lies within the FP32 error bound of its threshold
the oracle enumerates both ways and the GPU pixel must equal one of the outcomes; gradients are compared
with the oracle's for the outcomes the GPU took (tests/parity.py). Each check prints its share of such
pixels and of gradient elements that needed the error-scale term.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import binning  # noqa: E402
from paper_2603_02887_gb300 import synth  # noqa: E402
from paper_2603_02887_gb300.render import Renderer, render  # noqa: E402
from tests import parity  # noqa: E402
from tests.gpu_util import frame_arrays, upload  # noqa: E402

MODELS = ["exp", "sub", "lin", "sup"]
NT = os.cpu_count() or 4
KC = -0.5 * 1.4426950408889634  # conic scale folded into the records


@pytest.fixture(scope="module")
def rnd():
    r = Renderer("cuda:0")
    yield r
    r.close()


def _records_to_oracle_layout(rec):
    rec = rec.astype(np.float64)  # the FP32 record values, exactly
    return dict(u=rec[:, 0], v=rec[:, 1], A=rec[:, 2] / KC, B=rec[:, 3] / (2 * KC), C=rec[:, 4] / KC,
                aleph=np.exp2(rec[:, 5].astype(np.float64)), E=rec[:, [6, 7, 8]], z=rec[:, 9], rx=rec[:, 10],
                ry=rec[:, 11])


@pytest.mark.parametrize("which", ["tiny", "clustered"])
def test_projection_matches_oracle(rnd, which):
    if which == "tiny":
        scene, cam = synth.tiny_scene(0), synth.tiny_camera()
    else:
        scene, cam = synth.clustered_scene(4000, seed=1, sh_degree=3), synth.outside_camera(640, 360)
    params = upload(scene)
    _, _, frame = rnd.render(params, cam, "sup")
    fa = frame_arrays(frame)
    g = _records_to_oracle_layout(fa["records"])
    ref = oracle.project(scene, cam)
    live = fa["records"][:, 10] > 0
    assert np.array_equal(live, ref["valid"]), "valid set differs"
    rr = ref["rec"][live]
    np.testing.assert_allclose(g["u"][live], rr[:, 0], rtol=2e-6, atol=2e-4)
    np.testing.assert_allclose(g["v"][live], rr[:, 1], rtol=2e-6, atol=2e-4)
    scale = np.maximum(np.abs(rr[:, 2]), np.abs(rr[:, 4]))
    for j, key in ((2, "A"), (3, "B"), (4, "C")):
        assert np.all(np.abs(g[key][live] - rr[:, j]) <= 2e-4 * scale), key
    np.testing.assert_allclose(g["aleph"][live], rr[:, 5], rtol=2e-6)
    np.testing.assert_allclose(g["E"][live], rr[:, 6:9], atol=2e-5)
    assert np.array_equal(g["z"].astype(np.float32), ref["z32"]), "FP32 sort depth must be bit-identical"
    # the bounding box of the alpha >= alpha_min ellipse: half extents sqrt(tau Sigma'_xx), sqrt(tau Sigma'_yy)
    det = rr[:, 2] * rr[:, 4] - rr[:, 3] ** 2
    tau = 2 * np.log(rr[:, 5] / np.float32(1 / 255.0))
    assert np.all(g["rx"][live] >= np.sqrt(tau * rr[:, 4] / det)), "bounding box must be conservative"
    assert np.all(g["ry"][live] >= np.sqrt(tau * rr[:, 2] / det)), "bounding box must be conservative"
    # the FP32 error model behind the oracle's borderline decisions holds for the GPU's own records:
    # (u, v) within pos_err, the conic within 16 u relative (B: 16 u sqrt(A C)), L = log2(aleph) within
    # (8 + 4 |L|) u, the colour channels within e_band; each widened by the oracle's safety factor 2
    u = 2.0 ** -24
    pe = ref["pos_err"][live]
    assert np.all(np.abs(g["u"][live] - rr[:, 0]) <= 2 * pe[:, 0]), np.max(np.abs(g["u"][live] - rr[:, 0]) / pe[:, 0])
    assert np.all(np.abs(g["v"][live] - rr[:, 1]) <= 2 * pe[:, 1]), np.max(np.abs(g["v"][live] - rr[:, 1]) / pe[:, 1])
    sq = np.sqrt(rr[:, 2] * rr[:, 4])
    for j, key, sc in ((2, "A", rr[:, 2]), (3, "B", sq), (4, "C", rr[:, 4])):
        ratio = np.abs(g[key][live] - rr[:, j]) / (32 * u * sc)
        assert np.all(ratio <= 1), (key, float(ratio.max()))
    L = np.log2(rr[:, 5])
    rec_L = fa["records"][live, 5].astype(np.float64)
    assert np.all(np.abs(rec_L - L) <= 2 * u * (8 + 4 * np.abs(L))), float(np.max(np.abs(rec_L - L) / (u * (8 + 4 * np.abs(L)))))
    eb = ref["e_band"][live]
    e64 = np.maximum(rr[:, 6:9], 0)
    assert np.all(np.abs(g["E"][live] - e64) <= eb), float(np.max(np.abs(g["E"][live] - e64) / eb))


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (16, 32)])
def test_binning_keys_bit_exact(rnd, tile):
    scene, cam = synth.clustered_scene(3000, seed=2, sh_degree=1), synth.outside_camera(333, 211)
    params = upload(scene)
    _, _, frame = rnd.render(params, cam, "exp", options=dict(tile_w=tile[0], tile_h=tile[1]))
    fa = frame_arrays(frame)
    keys, vals, ranges = binning.sorted_pairs(fa["records"], fa["view"]["log2_alpha_min"], tile[0], tile[1],
                                              cam["width"], cam["height"])
    assert fa["view"]["n_pairs"] == len(keys)
    assert np.array_equal(fa["keys"], keys)
    assert np.array_equal(fa["values"], vals)
    assert np.array_equal(fa["ranges"].astype(np.int64), ranges)


def _oracle_opts(options):
    return options and {k: v for k, v in options.items() if k not in ("tile_w", "tile_h", "chunk", "schedule")}


def _forward_check(rnd, scene, cam, model, options=None, label=""):
    """Every pixel equals one of the oracle's outcomes for it (image max-abs 1e-4, overdraw exact)."""
    params = upload(scene)
    image, overdraw, frame = rnd.render(params, cam, model, options)
    ref = oracle.render(scene, cam, model, opts=_oracle_opts(options), nthreads=NT, outcomes=True)
    m = parity.assert_forward(image.cpu().numpy(), overdraw.cpu().numpy(), ref, label=f"{label} {model}")
    assert m.n_unresolved == 0, m.summary()
    print(f"[parity] forward {label} {model}: {m.summary()}")
    return image, overdraw, frame, ref


@pytest.mark.parametrize("model", MODELS)
def test_forward_matches_oracle_tiny(rnd, model):
    _forward_check(rnd, synth.tiny_scene(0), synth.tiny_camera(), model)


@pytest.mark.parametrize("model", MODELS)
def test_forward_matches_oracle_clustered_ragged(rnd, model):
    """Several tiles and a ragged tail in both directions, SH degree 3, an oblique camera."""
    _forward_check(rnd, synth.clustered_scene(20000, seed=4, sh_degree=3), synth.outside_camera(203, 141, 12.0),
                   model)


def test_tile_shapes_bit_identical(rnd):
    scene, cam = synth.clustered_scene(20000, seed=5, sh_degree=2), synth.outside_camera(250, 170, 13.0)
    params = upload(scene)
    for model in MODELS:
        outs = []
        for tile in ((8, 8), (16, 16), (16, 32)):
            img, od, _ = rnd.render(params, cam, model, dict(tile_w=tile[0], tile_h=tile[1]))
            outs.append((img.cpu().numpy(), od.cpu().numpy()))
        for img, od in outs[1:]:
            assert np.array_equal(img, outs[0][0]) and np.array_equal(od, outs[0][1]), model


def _backward_check(rnd, scene, cam, model, seed=3, options=None, label=""):
    """Forward as _forward_check, then the path-replay gradients against the oracle's for the outcomes the
    GPU took, every Gaussian included."""
    params = upload(scene)
    image, overdraw, frame = rnd.render(params, cam, model, options)
    g = synth.upstream_gradient(cam["height"], cam["width"], seed=seed)
    ref = oracle.render(scene, cam, model, opts=_oracle_opts(options), nthreads=NT, dl_dimage=g.astype(np.float64),
                        outcomes=True)
    m = parity.assert_forward(image.cpu().numpy(), overdraw.cpu().numpy(), ref, label=f"{label} {model}")
    assert m.n_unresolved == 0, m.summary()
    grads = rnd.backward(frame, params, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    rep = parity.assert_gradients({k: v.cpu().numpy() for k, v in grads.items()}, ref, m, label=f"{label} {model}")
    print(f"[parity] backward {label} {model}: {m.summary()}; {rep.summary()}")
    return grads, ref


@pytest.mark.parametrize("model", MODELS)
def test_backward_matches_oracle_tiny(rnd, model):
    _backward_check(rnd, synth.tiny_scene(0), synth.tiny_camera(), model)


@pytest.mark.parametrize("model", MODELS)
def test_backward_matches_oracle_clustered(rnd, model):
    _backward_check(rnd, synth.clustered_scene(6000, seed=6, sh_degree=3), synth.outside_camera(160, 120, 12.0),
                    model)


@pytest.mark.parametrize("model", MODELS)
def test_backward_matches_oracle_bench_options(rnd, model):
    """The replay in the launch configuration bench.py times for this model (bench.TUNED_OPTIONS:
    exponential on 8x8 tiles, the quadratic models on 16x16), on a scene spanning many tiles."""
    import bench
    _backward_check(rnd, synth.clustered_scene(6000, seed=8, sh_degree=3), synth.outside_camera(150, 110, 12.0),
                    model, options=bench.parse_options()[model])


def test_forward_is_deterministic(rnd):
    scene, cam = synth.clustered_scene(20000, seed=7, sh_degree=3), synth.outside_camera(300, 200)
    params = upload(scene)
    a = rnd.render(params, cam, "exp")[0].cpu().numpy()
    b = rnd.render(params, cam, "exp")[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_edge_cases(rnd):
    cam = synth.tiny_camera()
    # no Gaussians: background everywhere, no overdraw
    empty = {k: v[:0] for k, v in synth.tiny_scene(0).items()}
    img, od, _ = rnd.render(upload(empty), cam, "sup", dict(background=(0.25, 0.5, 0.75)))
    assert np.allclose(img.cpu().numpy(), [0.25, 0.5, 0.75]) and not od.cpu().numpy().any()
    # every Gaussian behind the camera
    behind = synth.tiny_scene(0)
    behind["means"] = behind["means"] * np.float32([1, 1, -1])
    img, od, _ = rnd.render(upload(behind), cam, "exp")
    assert not img.cpu().numpy().any() and not od.cpu().numpy().any()
    # one Gaussian covering the whole image, with a background
    one = synth.tiny_scene(0, n=1)
    one["means"][:] = [0.0, 0.0, 3.0]
    one["log_scales"][:] = 0.0
    for model in MODELS:  # one large splat: its alpha_min and alpha_max contours cross many pixels
        _forward_check(rnd, one, cam, model, dict(background=(0.2, 0.5, 0.9)), label="one splat")
    # ragged image smaller than one tile
    small = synth.pinhole(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 13, 7, 20.0, 20.0)
    for model in MODELS:
        _forward_check(rnd, synth.tiny_scene(1, n=200), small, model)


@pytest.mark.parametrize("model", ["exp", "sup"])
def test_maximum_image_width(rnd, model):
    """The largest accepted image side (16384 px) with a ragged last tile row: a 16384 x 21 frame against
    the oracle on windows at both ends and the middle; and 16385 is refused."""
    from paper_2603_02887_gb300._abi import NGSError

    cam = synth.pinhole(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 16384, 21, 3000.0, 3000.0)
    scene = synth.tiny_scene(5, n=4000)
    scene["means"][:, 0] *= 8.0  # spread across the wide frame, past both ends
    params = upload(scene)
    image, overdraw, _ = rnd.render(params, cam, model)
    img, od = image.cpu().numpy(), overdraw.cpu().numpy()
    assert od.sum() > 0
    for x0 in (0, 8192 - 32, 16384 - 64):
        win = (x0, 0, 64, 21)
        ref = oracle.render(scene, cam, model, window=win, nthreads=NT, outcomes=True)
        m = parity.assert_forward(img[:, x0:x0 + 64], od[:, x0:x0 + 64], ref, label=f"{model} x0={x0}")
        assert m.n_unresolved == 0
    with pytest.raises(NGSError):
        rnd.render(params, dict(cam, width=16385), model)


@pytest.mark.parametrize("model", MODELS)
def test_max_splats_cap(rnd, model):
    _forward_check(rnd, synth.tiny_scene(2), synth.tiny_camera(), model, dict(max_splats=3))


def test_invalid_arguments_are_rejected(rnd):
    from paper_2603_02887_gb300._abi import NGSError

    params = upload(synth.tiny_scene(0, n=10))
    cam = synth.tiny_camera()
    with pytest.raises(NGSError):
        rnd.render(params, cam, ("quad", -0.75))
    with pytest.raises(NGSError):
        rnd.render(params, cam, "sup", dict(tile_w=12, tile_h=12))
    with pytest.raises(NGSError):
        rnd.render(params, dict(cam, width=0), "sup")


def test_autograd_function_matches_direct_backward(rnd):
    """The autograd path and ngs_render_backward run the same kernels on the same frame data; only the
    order of their float atomics may differ. Both are held to the oracle for the outcomes the GPU took."""
    scene, cam = synth.tiny_scene(3, n=500), synth.tiny_camera()
    params = upload(scene)
    leaf = {k: v.clone().requires_grad_(True) for k, v in params.items()}
    image, overdraw = render(leaf, cam, "lin", renderer=rnd)
    g = torch.from_numpy(synth.upstream_gradient(128, 128, seed=9)).cuda()
    (image * g).sum().backward()
    _, od, frame = rnd.render(params, cam, "lin")
    direct = rnd.backward(frame, params, g)
    ref = oracle.render(scene, cam, "lin", nthreads=NT, dl_dimage=g.cpu().numpy().astype(np.float64), outcomes=True)
    m = parity.assert_forward(image.detach().cpu().numpy(), od.cpu().numpy(), ref)
    gref = parity.reference_gradients(ref, m)
    for name, grads in (("autograd", {k: leaf[k].grad.cpu().numpy() for k in params}),
                        ("direct", {k: direct["d_" + k].cpu().numpy() for k in params})):
        rep = parity.compare_gradients(grads, gref)
        assert rep.failed == 0 and rep.scaled <= 1e-3 * rep.n, (name, rep.summary(), rep.details)
    for k in params:
        # and with each other up to the order of the float additions: reordering a sum of N FP32 terms moves
        # it by at most (N - 1) u sum|terms|; the oracle's s_* is that sum chained to the parameters, and
        # N stays below 1600 (pixels hitting one splat on this frame), so 1e-4 s bounds the difference
        a, b = leaf[k].grad.cpu().numpy(), direct["d_" + k].cpu().numpy()
        s = ref["s_" + k].reshape(a.shape)
        assert np.all(np.abs(a - b) <= 1e-4 * s + 1e-12), k
