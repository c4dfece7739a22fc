"""Pins of the oracle's projection, per-pixel rendering and gradients (no GPU)."""
import math

import numpy as np
import pytest

from paper_2603_02887_gb300 import synth

MODELS = ["exp", "sub", "lin", "sup"]


def _one(mean, log_scale, quat, logit=2.0, sh=None):
    return dict(means=np.array([mean], np.float32), log_scales=np.array([log_scale], np.float32),
                quats=np.array([quat], np.float32), opacity_logits=np.array([logit], np.float32),
                sh=np.zeros((1, 1, 3), np.float32) if sh is None else np.asarray(sh, np.float32)[None])


def test_isotropic_on_axis_projection(orc):
    """An isotropic Gaussian of scale s on the optical axis at depth z projects to the image centre with
    2D covariance (f s / z)^2 I + dilation I, hence conic I / ((f s / z)^2 + 0.3)."""
    cam = synth.tiny_camera()
    s, z = 0.05, 4.0
    sc = _one([0, 0, z], [math.log(s)] * 3, [0.3, -0.2, 0.5, 0.7])
    p = orc.project(sc, cam)
    rec = p["rec"][0]
    s = math.exp(float(np.float32(math.log(s))))  # the parameter is stored in FP32
    var = (150.0 * s / z) ** 2 + float(np.float32(0.3))
    np.testing.assert_allclose(rec[:2], [64.0, 64.0], atol=1e-12)
    np.testing.assert_allclose(rec[2:5], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec[5], 1 / (1 + math.exp(-2.0)), rtol=1e-14)
    # degree-0 colour is constant: 0.5 + Y00 * 0 = 0.5 in every channel
    np.testing.assert_allclose(rec[6:9], 0.5, atol=0)
    assert p["valid"][0] and p["z32"][0] == np.float32(z)


def test_projection_against_independent_construction(orc):
    """Screen covariance J W Sigma W^T J^T + 0.3 I built independently: rotation matrix from scipy's
    quaternion routine, J as the numerical Jacobian of the pinhole map."""
    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng(7)
    cam = synth.outside_camera(320, 200)
    sc = synth.clustered_scene(64, seed=3, sh_degree=1)
    p = orc.project(sc, cam)
    V = np.asarray(cam["viewmat"], np.float32).astype(np.float64)
    R, t = V[:, :3], V[:, 3]
    fx, fy, cx, cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))

    def pix(pw):
        pv = R @ pw + t
        return np.array([fx * pv[0] / pv[2] + cx, fy * pv[1] / pv[2] + cy])

    checked = 0
    for g in range(64):
        if not p["valid"][g]:
            continue
        m = sc["means"][g].astype(np.float64)
        q = sc["quats"][g].astype(np.float64)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = np.diag(np.exp(sc["log_scales"][g].astype(np.float64)))
        Sig = Rq @ S @ S @ Rq.T
        h = 1e-6
        Jw = np.stack([(pix(m + h * e) - pix(m - h * e)) / (2 * h) for e in np.eye(3)], axis=1)  # d pix / d world
        S2 = Jw @ Sig @ Jw.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(S2)
        rec = p["rec"][g]
        np.testing.assert_allclose(rec[:2], pix(m), rtol=1e-12)
        np.testing.assert_allclose(rec[2:5], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6,
                                   atol=1e-9 * np.abs(conic).max())
        lam = np.linalg.eigvalsh(S2).max()
        aleph = 1 / (1 + math.exp(-float(sc["opacity_logits"][g])))
        a_min = float(np.float32(1 / 255.0))
        np.testing.assert_allclose(rec[9], math.sqrt(2 * math.log(aleph / a_min) * lam), rtol=1e-6)
        checked += 1
    assert checked > 40
    # the FP32 sort depth agrees with the exact view depth to FP32 rounding
    np.testing.assert_allclose(p["z32"], (sc["means"].astype(np.float64) @ R[2] + t[2]), rtol=1e-6)


def test_sh_basis_orthonormal_by_quadrature(orc):
    """The degree-3 real SH basis used for emission is orthonormal on the sphere: Gauss-Legendre in
    cos(theta) x uniform phi, exact for the degree-6 products. Y_k is read back through the projection
    as (E - 1/2) / 0.1 with SH coefficients 0.1 e_k in the red channel."""
    nodes, weights = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * math.pi / 16
    dirs, w = [], []
    for ct, wt in zip(nodes, weights):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            dirs.append([st * math.cos(ph), st * math.sin(ph), ct])
            w.append(wt * 2 * math.pi / 16)
    dirs, w = np.array(dirs), np.array(w)
    K = 16
    Y = np.zeros((len(dirs), K))
    for k in range(K):
        sh = np.zeros((len(dirs), K, 3), np.float32)
        sh[:, k, 0] = 0.1
        sc = dict(means=(5.0 * dirs).astype(np.float32), log_scales=np.full((len(dirs), 3), -3, np.float32),
                  quats=np.tile(np.float32([1, 0, 0, 0]), (len(dirs), 1)),
                  opacity_logits=np.zeros(len(dirs), np.float32), sh=sh)
        for sign in (1.0, -1.0):  # two cameras at the origin, looking down +z and -z
            vm = np.zeros((3, 4))
            vm[:, :3] = np.diag([sign, 1.0, sign])
            cam = synth.pinhole(vm, 64, 64, 50.0, 50.0)
            p = orc.project(sc, cam)
            sel = p["valid"] & (sign * dirs[:, 2] > 0)
            # the direction is taken from the stored FP32 means; renormalise the reference accordingly
            Y[sel, k] = (p["rec"][sel, 6] - 0.5) / 0.1
    d32 = (5.0 * dirs).astype(np.float32).astype(np.float64)
    assert np.allclose(np.linalg.norm(d32, axis=1), 5.0, rtol=1e-6)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(K), atol=2e-6)


def test_complex_step_jacobian_matches_finite_differences(orc):
    """The projection Jacobian the oracle chains gradients through (complex step) against central
    differences of the real projection."""
    sc = synth.clustered_scene(40, seed=5, sh_degree=3)
    cam = synth.outside_camera(400, 300)
    p = orc.project(sc, cam)
    keys = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    checked = 0
    for g in np.nonzero(p["valid"])[0][:8]:
        jac = orc.project_jacobian(sc, cam, g)
        col = 0
        for key in keys:
            arr = sc[key]
            width = int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1
            for j in range(width):
                sp = {k: v.astype(np.float64) for k, v in sc.items()}
                sm = {k: v.astype(np.float64) for k, v in sc.items()}
                base = float(sp[key].reshape(len(arr), -1)[g, j])
                h = 1e-6 * max(1.0, abs(base))
                sp[key].reshape(len(arr), -1)[g, j] += h
                sm[key].reshape(len(arr), -1)[g, j] -= h
                fd = (orc.project(sp, cam)["rec"][g, :9] - orc.project(sm, cam)["rec"][g, :9]) / (2 * h)
                scale = np.maximum(np.abs(jac[:, col]), np.abs(fd)).max() + 1e-12
                np.testing.assert_allclose(jac[:, col], fd, atol=2e-6 * scale + 1e-9, rtol=2e-6)
                col += 1
                checked += 1
    assert checked > 400


def test_prefilter_equals_brute_force(orc):
    """The disc bound |d| <= sqrt(2 ln(aleph/alpha_min) lambda_max) drops only pixels with alpha < alpha_min."""
    sc = synth.tiny_scene(0, n=300)
    cam = synth.tiny_camera()
    for m in MODELS:
        a = orc.render(sc, cam, m, nthreads=4)
        b = orc.render(sc, cam, m, nthreads=4, brute_force=True)
        assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["overdraw"], b["overdraw"])
        assert np.array_equal(a["n_listed"], b["n_listed"])


def test_window_equals_full_frame_region(orc):
    sc = synth.tiny_scene(0)
    cam = synth.tiny_camera()
    full = orc.render(sc, cam, "sup", nthreads=4)
    part = orc.render(sc, cam, "sup", nthreads=4, window=(30, 41, 50, 33))
    assert np.array_equal(part["image"], full["image"][41:74, 30:80])
    assert np.array_equal(part["overdraw"], full["overdraw"][41:74, 30:80])


def test_exponential_pixels_are_textbook_alpha_blending(orc):
    """At sampled pixels: collect every splat with alpha >= 1/255 from the oracle's own projected records,
    sort by (FP32 depth, index), blend with the back-to-front over operator (3DGS, Eq. gaussian_splatting)
    and the T_eps stop, and compare with the oracle's image."""
    sc = synth.tiny_scene(1)
    cam = synth.tiny_camera()
    p = orc.project(sc, cam)
    img = orc.render(sc, cam, "exp", nthreads=4)
    rng = np.random.default_rng(0)
    a_min = float(np.float32(1 / 255.0))
    for _ in range(60):
        x, y = rng.integers(0, 128, 2)
        px, py = x + 0.5, y + 0.5
        rec = p["rec"]
        dx, dy = px - rec[:, 0], py - rec[:, 1]
        q = rec[:, 2] * dx * dx + 2 * rec[:, 3] * dx * dy + rec[:, 4] * dy * dy
        alpha = np.minimum(float(np.float32(0.99)), rec[:, 5] * np.exp(-0.5 * q))
        idx = np.nonzero(p["valid"] & (alpha >= a_min))[0]
        idx = idx[np.lexsort((idx, p["z32"][idx]))]
        T, keep = 1.0, []
        for i in idx:  # the 3DGS stop: skip the rest once T would fall below 1e-4
            if T * (1 - alpha[i]) < float(np.float32(1e-4)):
                break
            keep.append(i)
            T *= 1 - alpha[i]
        L = np.zeros(3)
        for i in reversed(keep):
            L = rec[i, 6:9] * alpha[i] + (1 - alpha[i]) * L
        np.testing.assert_allclose(img["image"][y, x], L, atol=1e-12)
        assert img["overdraw"][y, x] == len(keep)


@pytest.mark.parametrize("model", MODELS + [(2, 0.5), (3, 0.5)])
def test_render_gradient_matches_finite_differences(orc, model):
    """Gradients of L = sum(g * image) w.r.t. raw parameters (mean, log-scale, quaternion, opacity logit,
    SH) against central differences of the FP64 render, on a reduced tiny scene. A sample is redrawn if
    any pixel's composited list, stop or clamp state differs between the two sides of the stencil."""
    sc = synth.clustered_scene(120, seed=11, sh_degree=2, box=3.0)
    sc["log_scales"] += 1.5
    cam = synth.outside_camera(64, 48, distance=6.0)
    rng = np.random.default_rng(12)
    g = rng.standard_normal((48, 64, 3))
    base = orc.render(sc, cam, model, nthreads=4, dl_dimage=g)
    names = {"means": "d_means", "log_scales": "d_log_scales", "quats": "d_quats",
             "opacity_logits": "d_opacity_logits", "sh": "d_sh"}
    live = np.nonzero(np.abs(base["d_opacity_logits"]) > 1e-3)[0]
    assert len(live) > 20
    checked = 0
    for _ in range(60):
        key = rng.choice(list(names))
        gi = int(rng.choice(live))
        flat = sc[key].reshape(len(sc[key]), -1)
        j = int(rng.integers(0, flat.shape[1]))
        th = float(flat[gi, j])
        h = 1e-5 * max(1.0, abs(th))
        outs = []
        for sgn in (1, -1):
            s2 = {k: v.astype(np.float64).copy() for k, v in sc.items()}
            s2[key].reshape(len(s2[key]), -1)[gi, j] = th + sgn * h
            outs.append(orc.render(s2, cam, model, nthreads=4))
        if not (np.array_equal(outs[0]["signature"], base["signature"])
                and np.array_equal(outs[1]["signature"], base["signature"])):
            continue
        fd = (np.sum(g * outs[0]["image"]) - np.sum(g * outs[1]["image"])) / (2 * h)
        an = base[names[key]].reshape(len(sc[key]), -1)[gi, j]
        assert abs(fd - an) <= 2e-5 * max(abs(fd), 1e-2), (key, gi, j, fd, an)
        checked += 1
    assert checked >= 30


def test_overdraw_order_of_models(orc):
    """On the tiny scene the faster-than-exponential models composite fewer splats (the paper's
    overdraw ordering sup < lin < sub < exp, Table 3)."""
    sc = synth.tiny_scene(0)
    cam = synth.tiny_camera()
    od = {m: orc.render(sc, cam, m, nthreads=4)["overdraw"] for m in MODELS}
    assert od["sup"].mean() < od["lin"].mean() < od["sub"].mean() < od["exp"].mean()
    assert np.all(od["sup"] <= od["lin"]) and np.all(od["lin"] <= od["sub"])
