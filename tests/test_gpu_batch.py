"""GPU: batched multi-view rendering (ngs_render_batch) against single-view renders and the oracle.

* bit identity: every view of a batch equals the render of its camera alone -- image, overdraw, replay
  state, splat records, and the per-tile lists (keys with the view's first global tile removed, values
  with the view's first record removed) -- for the four models and the three tile shapes, on cameras of
  uneven, ragged sizes, one of them looking away from the scene (a view with no splats);
* gradients: the backward of a batch is the gradient of the sum over its views: against the sum of the
  FP64 oracle's per-view gradients on the tiny scene (three views), and against the sum of the GPU's own
  single-view gradients on a clustered scene;
* edge cases: a batch of one view equals ngs_render; n_views outside 1..4096 is rejected.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer  # noqa: E402
from tests import parity  # noqa: E402
from tests.gpu_util import batch_arrays, frame_arrays, upload  # noqa: E402

MODELS = ["exp", "sub", "lin", "sup"]
NT = os.cpu_count() or 4
SMALL_SIZES = ((97, 61), (128, 128), (200, 113), (64, 40), (160, 90))


@pytest.fixture(scope="module")
def rnd():
    r = Renderer("cuda:0")
    yield r
    r.close()


@pytest.fixture(scope="module")
def clustered():
    scene = synth.clustered_scene(20000, seed=5, sh_degree=3)
    cams = synth.orbit_cameras(5, radius=12.0, seed=7, resolutions=SMALL_SIZES)
    away = synth.look_at(np.array([0.0, 0.0, -12.0]), np.array([0.0, 0.0, -30.0]), 72, 56)
    return scene, cams[:3] + [away] + cams[3:]


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (16, 32)])
@pytest.mark.parametrize("model", MODELS)
def test_batch_views_bit_identical_to_single(rnd, clustered, model, tile):
    scene, cams = clustered
    params = upload(scene)
    n = len(scene["means"])
    opts = dict(tile_w=tile[0], tile_h=tile[1])
    images, overdraw, frame = rnd.render_batch(params, cams, model, options=opts)
    imgs, ods = frame.split(images), frame.split(overdraw)
    ba = batch_arrays(frame)
    tile_of = (ba["keys"] >> np.uint64(32)).astype(np.int64)
    single_frame = rnd.frame()
    total_pairs = 0
    for v, cam in enumerate(cams):
        img1, od1, single_frame = rnd.render(params, cam, model, options=opts, frame=single_frame)
        assert torch.equal(imgs[v], img1), f"view {v}: image differs"
        assert torch.equal(ods[v], od1), f"view {v}: overdraw differs"
        sa = frame_arrays(single_frame)
        assert np.array_equal(_bits(ba["records"][v * n:(v + 1) * n]), _bits(sa["records"])), f"view {v}: records"
        p0, p1 = ba["pixel_base"][v], ba["pixel_base"][v + 1]
        assert np.array_equal(_bits(ba["state"][p0:p1]), _bits(sa["state"].reshape(-1, 8))), f"view {v}: state"
        t0, t1 = int(ba["tile_base"][v]), int(ba["tile_base"][v + 1])
        sel = (tile_of >= t0) & (tile_of < t1)
        assert np.array_equal(ba["keys"][sel] - (np.uint64(t0) << np.uint64(32)), sa["keys"]), f"view {v}: keys"
        assert np.array_equal(ba["values"][sel] - np.uint32(v * n), sa["values"]), f"view {v}: values"
        r = ba["ranges"][t0:t1].astype(np.int64)
        sr = sa["ranges"].astype(np.int64)
        assert np.array_equal(r[:, 1] - r[:, 0], sr[:, 1] - sr[:, 0]), f"view {v}: list lengths"
        for t in np.nonzero(r[:, 1] > r[:, 0])[0]:  # every (view, tile) list, entry by entry
            assert np.array_equal(ba["values"][r[t, 0]:r[t, 1]] - np.uint32(v * n),
                                  sa["values"][sr[t, 0]:sr[t, 1]]), f"view {v} tile {t}: list"
        total_pairs += sa["view"]["n_pairs"]
        if v == 3:  # the camera looking away from the scene
            assert sa["view"]["n_pairs"] == 0 and not torch.any(img1)
    assert total_pairs == ba["view"]["n_pairs"]
    rnd.recycle(single_frame)


def _tiny_views():
    c0 = synth.tiny_camera()
    c1 = synth.look_at(np.array([0.3, -0.2, 0.0]), np.array([0.0, 0.0, 4.0]), 96, 80, hfov_deg=50.0)
    c2 = synth.look_at(np.array([-0.4, 0.1, 0.2]), np.array([0.1, 0.0, 4.0]), 112, 72, hfov_deg=55.0)
    return [c0, c1, c2]


@pytest.mark.parametrize("model", MODELS)
def test_batch_gradient_is_sum_over_views_oracle(rnd, model):
    """Each view of a batch against the oracle (every pixel, tests/parity.py), and the batch gradient
    against the sum of the oracle's per-view gradients for the outcomes each view's pixels took."""
    scene = synth.tiny_scene(0)
    cams = _tiny_views()
    params = upload(scene)
    images, ods, frame = rnd.render_batch(params, cams, model)
    dls, refs = [], []
    for v, cam in enumerate(cams):
        H, W = cam["height"], cam["width"]
        g = synth.upstream_gradient(H, W, seed=20 + v)
        r = oracle.render(scene, cam, model, nthreads=NT, dl_dimage=g.astype(np.float64), outcomes=True)
        m = parity.assert_forward(frame.split(images)[v].cpu().numpy(), frame.split(ods)[v].cpu().numpy(), r,
                                  label=f"view {v}")
        assert m.n_unresolved == 0, m.summary()
        refs.append(parity.reference_gradients(r, m))
        dls.append(g.reshape(-1, 3))
    dl = torch.from_numpy(np.concatenate(dls)).cuda()
    grads = rnd.backward(frame, params, dl)
    rep = parity.assert_gradients({k: v.cpu().numpy() for k, v in grads.items()}, parity.sum_refs(refs), None,
                                  label=model)
    print(f"[parity] batch of 3 views {model}: {rep.summary()}")


@pytest.mark.parametrize("model", ["exp", "sup"])
def test_batch_gradient_is_sum_of_single_view_gradients(rnd, clustered, model):
    scene, cams = clustered
    params = upload(scene)
    images, _, frame = rnd.render_batch(params, cams, model)
    dl_views = [torch.from_numpy(synth.upstream_gradient(c["height"], c["width"], seed=40 + v)).cuda()
                for v, c in enumerate(cams)]
    grads = rnd.backward(frame, params, torch.cat([d.reshape(-1, 3) for d in dl_views]))
    total = {k: torch.zeros_like(grads[k], dtype=torch.float64) for k in grads}
    for v, cam in enumerate(cams):
        _, _, f1 = rnd.render(params, cam, model)
        g1 = rnd.backward(f1, params, dl_views[v])
        for k in total:
            total[k] += g1[k].double()
        rnd.recycle(f1)
    for k in total:
        a, b = grads[k].double(), total[k]
        tol = 1e-3 * torch.maximum(b.abs(), 1e-3 * b.abs().max()) + 1e-5 * b.abs().max()
        assert torch.all((a - b).abs() <= tol), (k, float(((a - b).abs() - tol).max()))


def test_batch_of_one_equals_render(rnd):
    scene, cam = synth.clustered_scene(5000, seed=3, sh_degree=2), synth.outside_camera(211, 157)
    params = upload(scene)
    for model in MODELS:
        img1, od1, f1 = rnd.render(params, cam, model)
        img2, od2, f2 = rnd.render_batch(params, [cam], model)
        assert torch.equal(img1.reshape(-1, 3), img2) and torch.equal(od1.reshape(-1), od2)
        g = torch.from_numpy(synth.upstream_gradient(157, 211, seed=1)).cuda()
        ga, gb = rnd.backward(f1, params, g), rnd.backward(f2, params, g)
        for k in ga:  # the same kernels; only the order of the replay's atomic additions may differ
            assert torch.allclose(ga[k], gb[k], rtol=1e-4, atol=1e-6 * float(ga[k].abs().max())), k
        rnd.recycle(f1)
        rnd.recycle(f2)


def test_batch_rejects_bad_view_counts(rnd):
    scene, cam = synth.tiny_scene(0), synth.tiny_camera()
    params = upload(scene)
    with pytest.raises(ValueError):
        rnd.render_batch(params, [], "exp")
    with pytest.raises(_abi.NGSError, match="n_views"):
        rnd.render_batch(params, [synth.pinhole(cam["viewmat"], 4, 4, 10.0, 10.0)] * 4097, "exp")


@pytest.mark.parametrize("model", ["exp", "sup"])
@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (16, 32)])
def test_chunk_and_schedule_do_not_change_results(rnd, clustered, model, tile):
    """Every staging chunk (tile pixels x 1/2, 1, 2) and both schedules (one CTA per tile; persistent CTAs
    over the tiles by descending pair count) give bit-identical images, overdraw and replay state, and
    gradients equal up to the order of the replay's atomic additions."""
    scene, cams = clustered
    params = upload(scene)
    P = tile[0] * tile[1]
    dl = None
    ref = None
    for chunk in (P // 2, P, 2 * P):
        for schedule in ("tiles", "persistent"):
            opts = dict(tile_w=tile[0], tile_h=tile[1], chunk=chunk, schedule=schedule)
            img, od, frame = rnd.render_batch(params, cams, model, options=opts)
            st = batch_arrays(frame)["state"]
            if dl is None:
                dl = torch.from_numpy(synth.upstream_gradient(1, img.shape[0], seed=9).reshape(-1, 3)).cuda()
            g = rnd.backward(frame, params, dl)
            if ref is None:
                ref = (img.clone(), od.clone(), st, {k: v.clone() for k, v in g.items()})
                continue
            assert torch.equal(img, ref[0]) and torch.equal(od, ref[1]), (chunk, schedule)
            assert np.array_equal(st.view(np.uint32), ref[2].view(np.uint32)), (chunk, schedule)
            for k, v in g.items():
                r = ref[3][k]
                assert torch.allclose(v, r, rtol=1e-4, atol=1e-6 * float(r.abs().max())), (chunk, schedule, k)
            rnd.recycle(frame)


def test_invalid_chunk_and_schedule_rejected(rnd):
    scene, cam = synth.tiny_scene(0), synth.tiny_camera()
    params = upload(scene)
    with pytest.raises(_abi.NGSError, match="chunk"):
        rnd.render(params, cam, "exp", options=dict(chunk=100))
    with pytest.raises(_abi.NGSError, match="schedule"):
        rnd.render(params, cam, "exp", options=dict(schedule=7))


def test_graph_replay_bit_identical_and_reused(clustered):
    """With CUDA graphs on, renders equal the direct launches bit for bit; a new pose of the same sizes is a
    replay (no capture); a pair count above the captured capacity makes a new phase-2 capture."""
    scene, cams = clustered
    params = upload(scene)
    direct, graphed = Renderer("cuda:0"), Renderer("cuda:0")
    graphed.set_graphs(True)
    try:
        fd, fg = direct.frame(), graphed.frame()
        for model in ("exp", "sup"):
            for schedule in ("tiles", "persistent"):
                opts = dict(schedule=schedule)
                a = direct.render_batch(params, cams, model, options=opts, frame=fd)
                b = graphed.render_batch(params, cams, model, options=opts, frame=fg)
                assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), (model, schedule)
        # same sizes, other poses: replays only
        img = torch.empty_like(a[0])
        od = torch.empty_like(a[1])
        graphed.render_batch(params, cams, "sup", frame=fg, images=img, overdraw=od)
        n0 = graphed.graph_captures()
        rng = np.random.default_rng(99)
        moved = []
        for c in cams:  # keep each view's size, change its pose
            d = rng.standard_normal(3)
            moved.append(synth.look_at(12.0 * d / np.linalg.norm(d), np.zeros(3), c["width"], c["height"]))
        for pose_set in (moved, cams):
            gi, go, _ = graphed.render_batch(params, pose_set, "sup", frame=fg, images=img, overdraw=od)
            di, do, _ = direct.render_batch(params, pose_set, "sup", frame=fd)
            assert torch.equal(gi, di) and torch.equal(go, do)
        assert graphed.graph_captures() == n0, "a new pose must not need a new capture"
        # single view: a camera facing away (no pairs) then one facing the scene (many): the pair count
        # outgrows the captured capacity, so phase 2 is captured anew
        far = synth.look_at(np.array([0.0, 0.0, -12.0]), np.array([0.0, 0.0, -30.0]), 320, 240)
        near = synth.outside_camera(320, 240)
        f1 = graphed.frame()
        graphed.render(params, far, "lin", frame=f1)
        n1 = graphed.graph_captures()
        gi, go, f1 = graphed.render(params, near, "lin", frame=f1)
        assert graphed.graph_captures() > n1
        di, do, _ = direct.render(params, near, "lin")
        assert torch.equal(gi, di) and torch.equal(go, do)
        g1 = graphed.backward(f1, params, torch.ones_like(gi))
        d1 = direct.backward(direct.render(params, near, "lin")[2], params, torch.ones_like(di))
        for k in g1:
            assert torch.allclose(g1[k], d1[k], rtol=1e-4, atol=1e-6 * float(d1[k].abs().max())), k
    finally:
        direct.close()
        graphed.close()


def test_autotune_returns_a_valid_fastest_configuration(rnd, clustered):
    scene, cams = clustered
    params = upload(scene)
    best, table = rnd.autotune(params, cams, "sup", backward=True, reps=2)
    assert len(table) == 18  # 3 tile shapes x 3 chunks x 2 schedules
    assert {(t[0], t[1]) for t in table} == {(8, 8), (16, 16), (16, 32)}
    assert all(t[4] > 0 for t in table)
    fastest = min(table, key=lambda t: t[4])
    assert (best["tile_w"], best["tile_h"], best["chunk"], best["schedule"]) == fastest[:4]
    a = rnd.render_batch(params, cams, "sup")
    b = rnd.render_batch(params, cams, "sup", options=best)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
