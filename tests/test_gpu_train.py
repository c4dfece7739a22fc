"""GPU: the training-step kernels against the FP64 oracle (oracle/train_ref.py), and a short reconstruction.

* loss: (1 - lambda) L1 + lambda (1 - SSIM) to 1e-6 relative and its gradient to 1e-5 of its largest
  entry, on ragged image sizes (border windows) and lambda in {0, 0.2, 1};
* Adam: one and several steps, bounded and not, against the oracle's updates (FP32 vs FP64);
* split / prune: same survivors and children, in the same order, as the oracle (with the cap);
* a training run on synthetic targets: the loss falls and the densification keeps the arrays consistent.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import train_ref as T  # noqa: E402
from paper_2603_02887_gb300 import synth  # noqa: E402
from paper_2603_02887_gb300.render import PARAM_KEYS, Renderer  # noqa: E402
from paper_2603_02887_gb300.train import Adam, Trainer, densify, l1_ssim, psnr, render_targets  # noqa: E402
from tests.gpu_util import upload  # noqa: E402


@pytest.fixture(scope="module")
def rnd():
    r = Renderer("cuda:0")
    yield r
    r.close()


@pytest.mark.parametrize("size", [(37, 23), (128, 96), (301, 77)])
@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_matches_oracle(rnd, size, lam):
    W, H = size
    rng = np.random.default_rng(W * 7 + H)
    x = rng.random((H, W, 3)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32)
    (L, l1, ssim), dl = l1_ssim(rnd, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), lam)
    Lr, l1r, ssimr, gr = T.l1_ssim(x.astype(np.float64), y.astype(np.float64), lam)
    assert abs(L - Lr) <= 1e-6 * max(1.0, abs(Lr)) and abs(l1 - l1r) <= 1e-6 and abs(ssim - ssimr) <= 1e-6
    g = dl.cpu().numpy()
    assert np.abs(g - gr).max() <= 1e-5 * np.abs(gr).max() + 1e-12


@pytest.mark.parametrize("bounded", [True, False])
def test_adam_matches_oracle(rnd, bounded):
    rng = np.random.default_rng(5)
    n = 777
    p = {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
         "quats": rng.standard_normal((n, 4)), "opacity_logits": rng.normal(0, 1, n),
         "sh": rng.standard_normal((n, 16, 3)) * 0.1}
    pt = {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in p.items()}
    lr = (1e-2, 5e-3, 1e-3, 5e-2, 2.5e-3)
    adam = Adam(pt, lr=lr, bounded=bounded)
    ref = {k: (p[k].astype(np.float32).astype(np.float64), np.zeros(p[k].shape), np.zeros(p[k].shape)) for k in p}
    for t in range(1, 6):
        g = {k: rng.standard_normal(p[k].shape).astype(np.float32) for k in p}
        adam.step(rnd, pt, {"d_" + k: torch.from_numpy(g[k]).cuda() for k in p}, lr_scale=0.5)
        for i, k in enumerate(PARAM_KEYS):
            ref[k] = T.adam_step(*ref[k][:1], g[k], *ref[k][1:], lr=lr[i] * 0.5, t=t, eps=1e-15, bounded=bounded)
        for k in p:
            np.testing.assert_allclose(pt[k].cpu().numpy(), ref[k][0], rtol=2e-6, atol=2e-6 * max(lr))


def test_densify_matches_oracle(rnd):
    rng = np.random.default_rng(6)
    n = 3000
    p = {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-4, 1.5, (n, 3)),
         "quats": rng.standard_normal((n, 4)), "opacity_logits": rng.normal(-1, 3, n),
         "sh": rng.standard_normal((n, 4, 3))}
    p = {k: v.astype(np.float32) for k, v in p.items()}
    m = {k: rng.standard_normal(v.shape).astype(np.float32) for k, v in p.items()}
    vv = {k: rng.random(v.shape).astype(np.float32) for k, v in p.items()}
    accum = (rng.random(n) * 2e-3).astype(np.float32)
    count = rng.integers(0, 4, n).astype(np.float32)
    pt = {k: torch.from_numpy(v).cuda() for k, v in p.items()}
    adam = Adam(pt)
    adam.m = {k: torch.from_numpy(v).cuda() for k, v in m.items()}
    adam.v = {k: torch.from_numpy(v).cuda() for k, v in vv.items()}
    cap = 3400
    out = densify(rnd, pt, adam, torch.from_numpy(accum).cuda(), torch.from_numpy(count).cuda(), grad_threshold=3e-4,
                  max_gaussians=cap)
    ro, rm, rv = T.densify({k: v.astype(np.float64) for k, v in p.items()}, m, vv, accum.astype(np.float64),
                           count.astype(np.float64), 3e-4, 0.008, 1e-4, cap)
    assert out["means"].shape[0] == len(ro["means"]) <= cap
    assert out["means"].shape[0] > n - 1000  # some pruned, some split
    for k in PARAM_KEYS:
        np.testing.assert_allclose(out[k].cpu().numpy().reshape(len(ro[k]), -1), ro[k].reshape(len(ro[k]), -1),
                                   rtol=1e-5, atol=1e-6, err_msg=k)
        np.testing.assert_allclose(adam.m[k].cpu().numpy().reshape(len(rm[k]), -1), rm[k].reshape(len(rm[k]), -1),
                                   rtol=0, atol=0, err_msg=k)


@pytest.fixture(scope="module")
def recon(rnd):
    gt = upload(synth.clustered_scene(6000, seed=21, sh_degree=1, box=4.0))
    cams = synth.orbit_cameras(6, radius=10.0, seed=22, resolutions=((160, 120),))
    targets = render_targets(rnd, gt, cams, "sup")
    init = {k: v.clone() for k, v in gt.items()}
    g = torch.Generator(device="cuda").manual_seed(3)
    init["means"] += 0.01 * torch.randn(init["means"].shape, device="cuda", generator=g)
    init["opacity_logits"] -= 1.0
    init["sh"] += 0.1 * torch.randn(init["sh"].shape, device="cuda", generator=g)
    return gt, cams, targets, init


@pytest.mark.parametrize("model", ["exp", "sup"])
def test_training_converges(rnd, recon, model):
    """Perturbed opacities, colours and positions are pulled back toward the targets (no densification)."""
    gt, cams, targets, init = recon
    if model != "sup":
        targets = render_targets(rnd, gt, cams, model)
    tr = Trainer(init, cams, targets, model=model, iters=200, densify_until=0, renderer=rnd)
    before = psnr(rnd, tr.params, cams, targets, model)
    for _ in range(200):
        tr.step()
    after = psnr(rnd, tr.params, cams, targets, model)
    assert after > before + 3.0, (before, after)


def test_training_with_densification(rnd, recon):
    """Split / prune inside the loop: the arrays and the Adam state stay consistent, the count changes, the
    loss at the end is below the loss at the start."""
    gt, cams, targets, init = recon
    tr = Trainer(init, cams, targets, model="sup", iters=250, densify_every=50, prune_every=100, densify_until=240,
                 grad_threshold=5e-4, coarse_to_fine=((0, 1),), renderer=rnd)
    first = tr.step(read_loss=True)["loss"]
    for _ in range(248):
        tr.step()
    last = tr.step(read_loss=True)
    n = tr.params["means"].shape[0]
    assert n != 6000
    assert all(v.shape[0] == n for v in tr.params.values()) and all(v.shape[0] == n for v in tr.adam.m.values())
    assert all(v.shape[0] == n for v in tr.adam.v.values()) and tr.accum.shape[0] == n
    assert np.isfinite(last["loss"]) and last["loss"] < first, (first, last["loss"])
