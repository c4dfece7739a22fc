"""Pins of the training-step oracle (no GPU): each checks the oracle against something other than its own
formulas -- identities of SSIM, a closed form on constant images, central differences of the loss, Adam's
closed-form first step and steady state, and the variance a split preserves."""
import numpy as np

from oracle import train_ref as T


def test_window_is_normalised_gaussian():
    g = T.gaussian_window()
    assert len(g) == 11 and abs(g.sum() - 1.0) < 1e-15
    assert np.allclose(g, g[::-1])
    assert abs(g[6] / g[5] - np.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


def test_ssim_identities():
    rng = np.random.default_rng(0)
    x = rng.random((17, 23, 3))
    y = rng.random((17, 23, 3))
    L, l1, ssim, grad = T.l1_ssim(x, x, 0.2)
    assert L == 0.0 and l1 == 0.0 and abs(ssim - 1.0) < 1e-15
    assert T.l1_ssim(x, y)[2] == T.l1_ssim(y, x)[2]  # symmetric
    assert -1.0 <= T.l1_ssim(x, y)[2] < 1.0


def test_ssim_of_constant_images_closed_form():
    """Away from the border every window sees constants a and b: no variance, so
    s = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x = np.full((30, 30, 3), a)
    y = np.full((30, 30, 3), b)
    s = T.ssim_map(x, y)
    expect = (2 * a * b + T.C1) / (a * a + b * b + T.C1)
    assert np.allclose(s[5:-5, 5:-5], expect, rtol=0, atol=1e-12)


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    x = rng.random((12, 9, 3))
    y = rng.random((12, 9, 3))
    L, _, _, grad = T.l1_ssim(x, y, 0.2)
    h = 1e-6
    for idx in [(0, 0, 0), (5, 4, 1), (11, 8, 2), (6, 0, 2), (3, 7, 0)] + [tuple(rng.integers((12, 9, 3))) for _ in range(10)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (T.l1_ssim(xp, y, 0.2)[0] - T.l1_ssim(xm, y, 0.2)[0]) / (2 * h)
        assert abs(fd - grad[idx]) < 1e-7, (idx, fd, grad[idx])


def test_adam_first_step_and_steady_state():
    """Bias correction makes the first step lr g / |g| (for |g| >> eps); a constant gradient keeps that step
    at every later step; the bound clips steps larger than lr."""
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    p1, m, v = T.adam_step(p, g, m, v, lr=0.01, t=1)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-9)
    p2 = p1
    for t in range(2, 50):
        prev = p2
        p2, m, v = T.adam_step(p2, g, m, v, lr=0.01, t=t)
        assert np.allclose(prev - p2, 0.01 * np.sign(g), rtol=1e-9)
    # momentum carried over a small second moment makes the unbounded step exceed lr; the bounded one stops
    m0, v0 = np.array([5.0]), np.array([1e-12])
    pu = T.adam_step(np.zeros(1), np.array([1.0]), m0, v0, lr=0.1, t=2, bounded=False)[0]
    pb = T.adam_step(np.zeros(1), np.array([1.0]), m0, v0, lr=0.1, t=2, bounded=True)[0]
    assert -pu[0] > 0.1 and -pb[0] == 0.1


def _params(n, rng, sh=3):
    return {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
            "quats": rng.standard_normal((n, 4)), "opacity_logits": rng.normal(0, 2, n),
            "sh": rng.standard_normal((n, sh, 3))}


def test_split_preserves_mean_and_axis_variance():
    rng = np.random.default_rng(2)
    p = _params(6, rng)
    zeros = {k: np.zeros_like(v) for k, v in p.items()}
    accum, count = np.full(6, 1.0), np.ones(6)
    out, om, ov = T.densify(p, zeros, zeros, accum, count, grad_threshold=0.5, min_opacity=0.0, min_scale=0.0,
                            max_gaussians=100)
    assert len(out["means"]) == 12
    for i in range(6):
        c = out["means"][2 * i:2 * i + 2]
        assert np.allclose(c.mean(axis=0), p["means"][i], atol=1e-12)  # the pair's centre is the parent's
        a = int(np.argmax(p["log_scales"][i]))
        r = T._rotation_column(p["quats"][i], a)
        sig = np.exp(p["log_scales"][i][a])
        child_sig = np.exp(out["log_scales"][2 * i][a])
        spread = np.dot(c[0] - p["means"][i], r) ** 2  # mixture variance along r: child var + offset^2
        assert abs(child_sig ** 2 + spread - sig ** 2) < 1e-12 * max(1.0, sig ** 2)


def test_prune_and_cap():
    rng = np.random.default_rng(3)
    p = _params(10, rng)
    p["opacity_logits"][:] = 3.0
    p["opacity_logits"][[1, 4]] = -10.0        # opacity below 0.008
    p["log_scales"][7] = -12.0                 # largest scale below 1e-4
    m = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    accum = np.zeros(10)
    count = np.ones(10)
    accum[[0, 2, 3, 5]] = 1.0                  # split candidates
    out, om, ov = T.densify(p, m, m, accum, count, 0.5, 0.008, 1e-4, max_gaussians=9)
    # 7 survivors, room for 2 of the 4 candidates (0 and 2, in index order)
    assert len(out["means"]) == 9
    keep = [i for i in range(10) if i not in (1, 4, 7)]
    assert np.allclose(out["opacity_logits"], [p["opacity_logits"][i] for i in [0, 0, 2, 2, 3, 5, 6, 8, 9]])
    # kept Gaussians carry their moments, children start from zero
    assert np.allclose(om["means"][4], m["means"][3]) and np.all(om["means"][:4] == 0)
    assert set(keep) == {0, 2, 3, 5, 6, 8, 9}
