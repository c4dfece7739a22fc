"""GPU: the native render server (ngs_server_*) -- continuous batching and admission by memory.

* every result is the same alone and in the mix: each request's image and overdraw map equal, bit for bit,
  a plain render of that request alone, although the server merged it with others into multi-view
  batches on several workers whose work overlapped on the device;
* batching happens: requests submitted while the workers are busy join shared batches;
* admission: with a budget smaller than any batch the oldest batch in flight still proceeds, so every
  request completes (counted as over-budget admissions), with the same images;
* a bad request fails alone: it is refused at submission, the requests around it still render.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_02887_gb300 import _abi, synth  # noqa: E402
from paper_2603_02887_gb300.render import Renderer  # noqa: E402
from paper_2603_02887_gb300.serve import Server  # noqa: E402
from tests.gpu_util import upload  # noqa: E402

MODELS = ["exp", "sub", "lin", "sup"]
SIZES = ((97, 61), (128, 128), (200, 113), (64, 40), (160, 90))


@pytest.fixture(scope="module")
def scenes():
    return [upload(synth.clustered_scene(20000, seed=5, sh_degree=3)),
            upload(synth.clustered_scene(50000, seed=6, sh_degree=1))]


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    cams = synth.orbit_cameras(n, radius=12.0, seed=seed, resolutions=SIZES)
    return [(int(rng.integers(0, 2)), cams[i], MODELS[int(rng.integers(0, 4))]) for i in range(n)]


def _serve(server, reqs, bursts):
    for chunk in np.array_split(np.arange(len(reqs)), bursts):
        for i in chunk:
            sc, cam, model = reqs[i]
            server.submit(sc, cam, model, tag=int(i))
    done = {}
    while len(done) < len(reqs):
        for c in server.poll(wait_ms=50):
            done[c["tag"]] = c
    return done


def _check_against_alone(scenes, reqs, done):
    r = Renderer("cuda:0")
    try:
        for i, (sc, cam, model) in enumerate(reqs):
            c = done[i]
            assert c["status"] == 0, (i, c["status"])
            assert c["submit_s"] <= c["start_s"] + 1e-6 <= c["done_s"] + 2e-6
            img, od, f = r.render(scenes[sc], cam, model)
            assert torch.equal(c["image"], img), f"request {i}: image differs from the render alone"
            assert torch.equal(c["overdraw"], od), f"request {i}: overdraw differs from the render alone"
            r.recycle(f)
    finally:
        r.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_results_same_alone_and_in_the_mix(scenes, graphs):
    reqs = _requests(48, seed=11)
    server = Server(workers=3, max_batch_views=8, graphs=graphs)
    try:
        ids = [server.add_scene(p) for p in scenes]
        assert ids == [0, 1]
        done = _serve(server, reqs, bursts=3)
        st = server.stats()
    finally:
        server.close()
    assert st["completed"] == 48 and st["submitted"] == 48
    assert st["batches"] < 48 and st["max_batch_views"] > 1, "requests that wait must be batched"
    assert max(c["batch_views"] for c in done.values()) <= 8
    _check_against_alone(scenes, reqs, done)


def test_admission_always_progresses_under_a_tiny_budget(scenes):
    reqs = _requests(16, seed=12)
    server = Server(workers=4, max_batch_views=4, mem_budget=1)
    try:
        for p in scenes:
            server.add_scene(p)
        done = _serve(server, reqs, bursts=1)
        st = server.stats()
    finally:
        server.close()
    assert st["completed"] == 16
    assert st["over_budget_admissions"] > 0
    assert st["reserved_bytes"] == 0, "every reservation is released"
    _check_against_alone(scenes, reqs, done)


def test_bad_request_fails_alone(scenes):
    server = Server(workers=2, max_batch_views=1)
    try:
        server.add_scene(scenes[0])
        with pytest.raises(_abi.NGSError):
            server.submit(5, synth.tiny_camera(), "exp")  # no such scene
        server.submit(0, synth.tiny_camera(), "exp", tag=100)
        with pytest.raises(_abi.NGSError):
            server.submit(0, dict(synth.tiny_camera(), fx=-1.0), "exp", tag=101)
        with pytest.raises(_abi.NGSError):
            server.submit(0, synth.tiny_camera(), ("quad", -0.75), tag=102)
        server.submit(0, synth.tiny_camera(), "sup", tag=103)
        done = {}
        while len(done) < 2:
            for c in server.poll(wait_ms=50):
                done[c["tag"]] = c
        assert sorted(done) == [100, 103] and all(c["status"] == 0 for c in done.values())
        assert server.last_error() == ""
    finally:
        server.close()
