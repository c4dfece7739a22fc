"""Pins of the oracle's compositing operator (no GPU).

Each test checks the oracle against something other than itself: numbers printed in the paper
(Fig. 2 and Fig. 3 data under tests/golden/), closed forms that follow from Table 1, the textbook
over operator, invariants of Sec. 4.3, and central finite differences for the adjoints.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# model name in the golden files -> (oracle kind, parameter)
MODELS = {"exp": (0, 0.0), "quad_c-0.5": (1, -0.5), "quad_c0": (1, 0.0), "quad_c0.5": (1, 0.5),
          "quad_c1": (1, 1.0), "blend_g0.5": (2, 0.5), "vicini_g0.5": (3, 0.5)}


def _read(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.setdefault(parts[0], []).append([float(v) for v in parts[1:]])
    return {k: np.array(v) for k, v in rows.items()}


def _tbar(res, n):
    """Discrete transmittance Tbar_i = 1 - sum_{j<i} pbar_j for i = 0..n (Eq. generalized_gaussian)."""
    return 1.0 - np.concatenate([[0.0], np.cumsum(res["pbar"][:n])])


@pytest.mark.parametrize("model", list(MODELS))
def test_fig2_transmittance_dots(orc, model):
    """Fig. 2: 100 splats of opacity 0.02; the blue dots are Tbar after n = 0, 5, ..., 100 splats."""
    dots = _read("fig2_transmittance_dots.txt")[model]
    res = orc.composite_list(np.full(100, 0.02), np.ones((100, 3)), MODELS[model])
    tb = _tbar(res, 100)
    n = np.rint(dots[:, 0] / 0.02).astype(int)
    np.testing.assert_allclose(np.maximum(tb[n], 0.0), dots[:, 1], rtol=0, atol=6e-9)


def _mother(model, tau):
    """Continuous mother transmittances of Table 1."""
    kind, p = MODELS[model]
    if kind == 0:
        return np.exp(-tau)
    if kind == 1:
        return np.maximum(1 - tau - 0.5 * p * tau ** 2, 0.0)
    if kind == 2:
        return np.maximum((1 - p) * (1 - tau) + p * np.exp(-tau), 0.0)
    return (1 - p) * np.maximum(1 - tau, 0.0) + p * np.exp(-tau)


@pytest.mark.parametrize("model", list(MODELS))
def test_fig2_mother_curves_match_table1(model):
    """The green curves of Fig. 2 are Table 1's mother functions (pins the reading of Table 1)."""
    curves = _read("fig2_mother_curves.txt")
    c = curves[model]
    np.testing.assert_allclose(_mother(model, c[:, 0]), c[:, 1], atol=2e-4)  # tau printed to 4 decimals
    d = curves["exp_dashed"]
    np.testing.assert_allclose(np.exp(-d[:, 0]), d[:, 1], atol=2e-4)


@pytest.mark.parametrize("model", list(MODELS))
def test_thin_stacks_converge_to_mother(orc, model):
    """Dense thin stacks (alpha = tau/n, n -> inf) converge to the continuous T(tau) at rate O(1/n)
    (Sec. 4.4 'Transmittance' evaluation; App. A for the exponential)."""
    tau = 1.5
    errs = []
    for n in (100, 1000, 10000):
        res = orc.composite_list(np.full(n, tau / n), np.ones((n, 3)), MODELS[model])
        errs.append(abs(max(_tbar(res, n)[-1], 0.0) - _mother(model, tau)))
    assert errs[2] < 3e-3
    assert errs[2] <= errs[1] + 1e-12 <= errs[0] + 1e-12


@pytest.mark.parametrize("c", [-0.5, 0.0, 0.5, 1.0])
def test_quadratic_saturates_at_finite_depth(orc, c):
    """T = [1 - tau - c/2 tau^2]_+ reaches zero at tau* = (sqrt(1 + 2c) - 1)/c (tau* = 1 at c = 0); a thin
    stack saturates at taubar -> tau*, and after saturation every pbar is 0 (Eq. nexp_p)."""
    n = 20000
    a = 3.0 / n
    res = orc.composite_list(np.full(n, a), np.ones((n, 3)), (1, c))
    assert res["saturated"]
    k = res["m"] - 1
    # exact discrete position: the first i whose slope term reaches Tbar_i, with
    # Tbar_i = 1 - i a - c/2 a^2 i (i - 1) before saturation (sum of Table 1's slope terms)
    i = np.arange(n)
    tbar = 1 - i * a - 0.5 * c * a * a * i * (i - 1)
    assert k == int(np.argmax(a * (1 + c * i * a) >= tbar))
    # continuum limit: k a -> tau*; the double root of (1 - tau/2)^2 at c = -1/2 converges as sqrt(a)
    tau_star = 1.0 if c == 0 else (math.sqrt(1 + 2 * c) - 1) / c
    assert abs(k * a - tau_star) < (2 * math.sqrt(a) if c == -0.5 else 1e-3)
    assert np.all(res["pbar"][k + 1:] == 0)
    assert abs(res["pbar"][: k + 1].sum() - 1.0) < 1e-12
    assert res["T_end"] == 0.0


def _fig3_check(orc, scene):
    d = _read(f"fig3_{scene}_contributions.txt")
    ex = d["exp"]
    worst = 0.0
    used = 0
    for model, spec in MODELS.items():
        ref = d[model]
        for j in range(ex.shape[0]):
            r, g, b = ex[j, 1:4]
            # invert the three opacities from the exponential curves: red = a_r, green = a_g (1 - a_r),
            # blue = a_b (1 - a_r)(1 - a_g) (Eq. gaussian_splatting); skip samples where that is singular
            if r >= 0.999 or g / (1 - r) >= 0.999:
                continue
            ar = r
            ag = g / (1 - ar)
            ab = b / ((1 - ar) * (1 - ag))
            res = orc.composite_list([ar, ag, ab], np.eye(3), spec)
            np.testing.assert_allclose(res["pbar"], ref[j, 1:4], atol=3e-6, err_msg=f"{model} x={ex[j, 0]}")
            np.testing.assert_allclose(res["pbar"].sum(), ref[j, 4], atol=4e-6)
            worst = max(worst, np.abs(res["pbar"] - ref[j, 1:4]).max())
            used += 1
    return used, worst


def test_fig3_concentric_contributions(orc):
    """Fig. 3 (a): from opacities inverted out of the exponential curves, every other model's printed
    per-Gaussian contributions are predicted to print precision, saturating samples included."""
    used, worst = _fig3_check(orc, "concentric")
    assert used > 800 and worst < 3e-6


def test_fig3_cyclic_contributions(orc):
    """Fig. 3 (b), anisotropic rotated Gaussians."""
    used, worst = _fig3_check(orc, "cyclic")
    assert used > 800 and worst < 3e-6


def test_fig3_saturating_sample(orc):
    """A sample where the sub-linear model saturates at the third Gaussian: its contribution is the
    remainder 1 - (pbar_r + pbar_g), not its slope term (Eq. nexp_p, i = k)."""
    d = _read("fig3_concentric_contributions.txt")
    ex = d["exp"][d["exp"][:, 0] == 204][0]
    ref = d["quad_c-0.5"][d["quad_c-0.5"][:, 0] == 204][0]
    ar = ex[1]
    ag = ex[2] / (1 - ar)
    ab = ex[3] / ((1 - ar) * (1 - ag))
    res = orc.composite_list([ar, ag, ab], np.eye(3), (1, -0.5))
    assert res["saturated"]
    assert ab * (1 - 0.5 * (ar + ag)) > 1 - res["pbar"][:2].sum()  # the slope term would overshoot
    np.testing.assert_allclose(res["pbar"][2], ref[3], atol=3e-6)


def _random_list(rng, n, amax=0.99):
    return rng.uniform(0.0, amax, n), rng.uniform(0.0, 1.0, (n, 3))


def test_exponential_is_textbook_over(orc):
    """Exponential model = standard 3DGS blending = the recursive over operator L_i = E_i a_i +
    (1 - a_i) L_{i+1} evaluated back to front (Eq. gaussian_splatting, App. B Eq. oi_3dgs)."""
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 40):
        a, E = _random_list(rng, n)
        bg = rng.uniform(0, 1, 3)
        L = bg.copy()
        for i in range(n - 1, -1, -1):
            L = E[i] * a[i] + (1 - a[i]) * L
        res = orc.composite_list(a, E, (0, 0.0), background=bg)
        np.testing.assert_allclose(res["color"], L, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(res["T_end"], np.prod(1 - a), rtol=1e-13)


@pytest.mark.parametrize("c", [-0.5, 0.0, 0.5, 1.0])
def test_quadratic_closed_form_and_order_independence(orc, c):
    """Before saturation, Tbar = 1 - taubar - c/2 (taubar^2 - sum a^2), a symmetric function of the
    opacities (sum of Table 1's slope terms), so it does not depend on the order of the list."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        n = int(rng.integers(1, 12))
        a = rng.uniform(0, 0.08, n)
        res = orc.composite_list(a, np.ones((n, 3)), (1, c))
        tau = a.sum()
        closed = 1 - tau - 0.5 * c * (tau ** 2 - (a ** 2).sum())
        if res["saturated"]:
            continue
        np.testing.assert_allclose(res["T_end"], closed, atol=1e-14)
        perm = rng.permutation(n)
        res2 = orc.composite_list(a[perm], np.ones((n, 3)), (1, c))
        np.testing.assert_allclose(res2["T_end"], res["T_end"], atol=1e-14)


@pytest.mark.parametrize("model", list(MODELS))
def test_physical_constraints(orc, model):
    """Sec. 4.3: Tbar in [0, 1], Tbar_0 = 1, non-increasing; the first contribution equals alpha_1."""
    rng = np.random.default_rng(3)
    for _ in range(30):
        n = int(rng.integers(1, 60))
        a, E = _random_list(rng, n, amax=rng.choice([0.1, 0.5, 0.99]))
        res = orc.composite_list(a, E, MODELS[model])
        tb = _tbar(res, n)
        assert tb[0] == 1.0
        assert np.all(tb >= -1e-15) and np.all(tb <= 1.0)
        assert np.all(np.diff(tb) <= 1e-15)
        assert abs(res["pbar"][0] - a[0]) < 1e-15


def test_quadratic_overdraw_monotone_in_c(orc):
    """For the same list, a larger c saturates no later (the slope terms grow with c)."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        n = int(rng.integers(1, 80))
        a, E = _random_list(rng, n, amax=0.3)
        ms = [orc.composite_list(a, E, (1, c))["m"] for c in (-0.5, 0.0, 0.5, 1.0)]
        assert ms == sorted(ms, reverse=True)


def test_exponential_teps_stop(orc):
    """The exponential model stops before the splat that would take T below T_eps."""
    a = np.full(50, 0.5)
    res = orc.composite_list(a, np.ones((50, 3)), (0, 0.0), t_eps=1e-4)
    # (1/2)^13 = 1.2e-4 >= 1e-4 > (1/2)^14
    assert res["m"] == 13
    assert abs(res["T_end"] - 0.5 ** 13) < 1e-15


def test_max_splats_cap(orc):
    a = np.full(50, 0.01)
    for spec in MODELS.values():
        res = orc.composite_list(a, np.ones((50, 3)), spec, max_splats=7)
        assert res["m"] == 7


@pytest.mark.parametrize("model", list(MODELS))
def test_list_adjoint_matches_finite_differences(orc, model):
    """dL0/dalpha_i and dL0/dE_i of the oracle's adjoint (App. C recursion for the quadratic family)
    against central differences of the forward, on lists that do and do not saturate, with a background."""
    spec = MODELS[model]
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(40):
        n = int(rng.integers(1, 25))
        a, E = _random_list(rng, n, amax=rng.choice([0.15, 0.6]))
        bg = rng.uniform(0, 1, 3)
        g = rng.standard_normal(3)
        t_eps = 1e-4
        res = orc.composite_list(a, E, spec, t_eps=t_eps, background=bg, g=g)
        h = 1e-7
        for i in range(n):
            ap, am = a.copy(), a.copy()
            ap[i] += h
            am[i] -= h
            rp = orc.composite_list(ap, E, spec, t_eps=t_eps, background=bg)
            rm = orc.composite_list(am, E, spec, t_eps=t_eps, background=bg)
            if rp["m"] != res["m"] or rm["m"] != res["m"] or rp["saturated"] != rm["saturated"]:
                continue  # a stop decision flips inside the stencil
            fd = (g @ rp["color"] - g @ rm["color"]) / (2 * h)
            assert abs(fd - res["dalpha"][i]) < 1e-6 * max(1.0, abs(fd)), (model, trial, i)
            for ch in range(3):
                Ep, Em = E.copy(), E.copy()
                Ep[i, ch] += h
                Em[i, ch] -= h
                fdE = (g @ orc.composite_list(a, Ep, spec, t_eps=t_eps, background=bg)["color"]
                       - g @ orc.composite_list(a, Em, spec, t_eps=t_eps, background=bg)["color"]) / (2 * h)
                assert abs(fdE - res["dE"][i, ch]) < 1e-6 * max(1.0, abs(fdE))
            checked += 1
    assert checked > 100
