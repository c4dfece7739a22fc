"""Pins of the oracle's enumeration of borderline decisions (no GPU).

Where a compositing decision's FP64 value lies within the FP32 error bound of its threshold, the oracle
enumerates both ways. Each test builds a list whose decision sits a hair (1e-9) from its threshold and
checks the enumerated outcomes against the plain operator (``composite_list``, pinned to the paper's
Fig. 2 / Fig. 3 data in test_oracle_composite.py) evaluated on inputs nudged to either side of that
threshold: an independent construction of the same two outcomes. The last tests pin the parity helper
itself with mistakes planted in a fake "GPU" result built from the oracle.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2603_02887_gb300 import synth
from tests import parity

E3 = np.array([[0.9, 0.1, 0.2], [0.1, 0.8, 0.3], [0.2, 0.3, 0.7], [0.5, 0.5, 0.1], [0.3, 0.6, 0.9]])
HAIR = 1e-9
BAND = 1e-6  # log2-domain bound given to every candidate: far wider than the hair, far narrower than
             # any other decision's distance in these lists


def _same(o, ref, atol=1e-7):
    return o["m"] == ref["m"] and np.allclose(o["color"], ref["color"], atol=atol) and \
        np.allclose(o["pbar"], ref["pbar"], atol=atol)


def _outcome_set_matches(outs, refs):
    """Each expected outcome appears among the enumerated ones, and each enumerated one is expected."""
    assert outs is not None
    assert len(outs) == len(refs), (len(outs), len(refs))
    for r in refs:
        assert any(_same(o, r) for o in outs), (r, outs)
    for o in outs:
        assert any(_same(o, r) for r in refs), (o, refs)


@pytest.mark.parametrize("c", [-0.5, 0.0, 0.5, 1.0])
def test_saturation_borderline(c):
    """S after entry 1 is 1 - 1e-9: the FP64 walk does not saturate there, the other outcome does."""
    a0 = 0.55
    a1 = (1.0 - HAIR - a0) / (1.0 + c * a0)
    alpha = np.array([a0, a1, 0.3, 0.2])
    outs = oracle.composite_outcomes(alpha, E3[:4], (1, c), band=BAND)
    assert outs[0]["m"] == 3  # FP64: entry 1 keeps S below 1, entry 2 saturates
    nudged = alpha.copy()
    nudged[1] = (1.0 + HAIR - a0) / (1.0 + c * a0)  # now entry 1 saturates in FP64
    refs = [oracle.composite_list(alpha, E3[:4], (1, c)), oracle.composite_list(nudged, E3[:4], (1, c))]
    _outcome_set_matches(outs, refs)


def test_blended_saturation_borderline():
    g = 0.5
    a0 = 0.6
    f1 = 1.0 - g + g * (1.0 - a0)
    a1 = (1.0 - HAIR - a0) / f1
    alpha = np.array([a0, a1, 0.4])
    outs = oracle.composite_outcomes(alpha, E3[:3], (2, g), band=BAND)
    nudged = alpha.copy()
    nudged[1] = (1.0 + HAIR - a0) / f1
    _outcome_set_matches(outs, [oracle.composite_list(alpha, E3[:3], (2, g)),
                                oracle.composite_list(nudged, E3[:3], (2, g))])


@pytest.mark.parametrize("model", [(0, 0.0), (1, -0.5), (1, 0.5)])
def test_alpha_min_borderline(model):
    """A candidate a hair above alpha_min: composited in FP64, skipped in the other outcome."""
    amin = 0.1
    raw = np.array([0.3, amin * 2 ** (HAIR), 0.2, 0.25])
    outs = oracle.composite_outcomes(raw, E3[:4], model, band=BAND, alpha_min=amin, t_eps=1e-4)
    keep = [oracle.composite_list(raw, E3[:4], model, t_eps=1e-4)]
    drop = oracle.composite_list(raw[[0, 2, 3]], E3[[0, 2, 3]], model, t_eps=1e-4)
    drop["pbar"] = np.insert(drop["pbar"], 1, 0.0)
    _outcome_set_matches(outs, keep + [drop])


def test_alpha_min_borderline_below():
    """A candidate a hair below alpha_min: skipped in FP64, composited in the other outcome."""
    amin = 0.1
    raw = np.array([0.3, amin * 2 ** (-HAIR), 0.2])
    outs = oracle.composite_outcomes(raw, E3[:3], (1, 0.0), band=BAND, alpha_min=amin)
    skip = oracle.composite_list(raw[[0, 2]], E3[[0, 2]], (1, 0.0))
    skip["pbar"] = np.insert(skip["pbar"], 1, 0.0)
    take = oracle.composite_list(raw, E3[:3], (1, 0.0))
    _outcome_set_matches(outs, [skip, take])
    assert outs[0]["m"] == 2


def test_alpha_max_borderline():
    """aleph K a hair above alpha_max: clamped in FP64, not in the other outcome."""
    amax = 0.9
    raw = np.array([0.2, amax * 2 ** HAIR, 0.3])
    outs = oracle.composite_outcomes(raw, E3[:3], (0, 0.0), band=BAND, alpha_max=amax)
    clamped = oracle.composite_list([0.2, amax, 0.3], E3[:3], (0, 0.0))
    free = oracle.composite_list(raw, E3[:3], (0, 0.0))
    _outcome_set_matches(outs, [clamped, free])


def test_teps_borderline():
    """T (1 - alpha_2) a hair above t_eps: the FP64 walk composites entry 2, the other stops before it."""
    teps = 1e-4
    alpha = np.array([0.9, 0.9, 0.0, 0.5])
    alpha[2] = 1.0 - teps * (1.0 + HAIR) / (0.1 * 0.1)
    outs = oracle.composite_outcomes(alpha, E3[:4], (0, 0.0), band=BAND, t_eps=teps)
    go = oracle.composite_list(alpha, E3[:4], (0, 0.0), t_eps=teps)
    stop = oracle.composite_list(alpha, E3[:4], (0, 0.0), t_eps=teps * (1.0 + 3 * HAIR))
    assert go["m"] == 3 and stop["m"] == 2
    _outcome_set_matches(outs, [go, stop])


def test_two_borderline_decisions():
    """A borderline alpha_min candidate before a borderline saturation: the outcomes are every
    combination that the walk can meet (skipping the candidate moves the sum away from saturation at
    entry 2, where no decision is borderline any more)."""
    amin = 0.05
    a0, a2 = 0.5, None
    a1 = amin * 2 ** HAIR
    a2 = 1.0 - HAIR - a0 - a1  # linear: S after entry 2 is 1 - 1e-9
    raw = np.array([a0, a1, a2, 0.3])
    outs = oracle.composite_outcomes(raw, E3[:4], (1, 0.0), band=BAND, alpha_min=amin)
    refs = []
    for take1, sat2 in itertools.product([True, False], [False, True]):
        lst = raw.copy()
        if sat2:
            lst[2] += 2 * HAIR
        idx = [0, 1, 2, 3] if take1 else [0, 2, 3]
        r = oracle.composite_list(lst[idx], E3[idx], (1, 0.0))
        if not take1:
            r["pbar"] = np.insert(r["pbar"], 1, 0.0)
        if take1 or not sat2:
            refs.append(r)
    # without candidate 1, S after entry 2 is 1 - amin - 1e-9: the saturation is not borderline there
    _outcome_set_matches(outs, refs)


def test_no_borderline_decision_gives_one_outcome():
    rng = np.random.default_rng(3)
    for kind in [(0, 0.0), (1, -0.5), (1, 0.0), (1, 0.5), (2, 0.5), (3, 0.5)]:
        for _ in range(20):
            n = int(rng.integers(1, 12))
            raw = rng.uniform(0.02, 0.6, n)
            E = rng.uniform(0, 1, (n, 3))
            outs = oracle.composite_outcomes(raw, E, kind, band=1e-13, t_eps=1e-4)
            assert len(outs) == 1
            ref = oracle.composite_list(raw, E, kind, t_eps=1e-4)
            assert _same(outs[0], ref, atol=0)


def test_error_bound_of_the_fp32_alpha_evaluation():
    """The oracle's bound on log2(alpha) covers an FP32 evaluation of the GPU's formula
    L + dx (A' dx + B' dy) + C' dy^2 from records rounded to FP32 with the screen position perturbed
    by its stated error bound: at sampled (splat, pixel) pairs of a clustered scene the FP32 value
    stays within the bound of the FP64 one wherever the pixel has a single outcome."""
    sc, cam = synth.clustered_scene(3000, seed=5, sh_degree=1), synth.outside_camera(200, 150)
    p = oracle.project(sc, cam)
    rec = p["rec"][p["valid"]]
    pos = p["pos_err"][p["valid"]]
    rng = np.random.default_rng(0)
    k = np.float32(-0.5 * 1.4426950408889634)
    worst = 0.0
    for sign in (1.0, -1.0):
        u32 = (rec[:, 0] + sign * pos[:, 0]).astype(np.float32)
        v32 = (rec[:, 1] - sign * pos[:, 1]).astype(np.float32)
        A32 = (k * rec[:, 2].astype(np.float32)).astype(np.float32)
        B32 = (np.float32(2) * k * rec[:, 3].astype(np.float32)).astype(np.float32)
        C32 = (k * rec[:, 4].astype(np.float32)).astype(np.float32)
        L32 = np.log2(rec[:, 5]).astype(np.float32)
        for _ in range(20):
            px = np.float32(rng.integers(0, 200) + 0.5)
            py = np.float32(rng.integers(0, 150) + 0.5)
            dx = px - u32
            dy = py - v32
            l32 = L32 + dx * (A32 * dx + B32 * dy) + C32 * dy * dy
            ddx, ddy = px - rec[:, 0], py - rec[:, 1]
            q = rec[:, 2] * ddx ** 2 + 2 * rec[:, 3] * ddx * ddy + rec[:, 4] * ddy ** 2
            l64 = np.log2(rec[:, 5]) - 0.5 * 1.4426950408889634 * q
            near = l64 > -12  # the region where decisions are taken
            Q = (np.sqrt(rec[:, 2]) * np.abs(ddx) + np.sqrt(rec[:, 4]) * np.abs(ddy)) ** 2
            posb = 1.4426950408889634 * (np.abs(rec[:, 2] * ddx + rec[:, 3] * ddy) * pos[:, 0] / 2 ** -24 +
                                         np.abs(rec[:, 3] * ddx + rec[:, 4] * ddy) * pos[:, 1] / 2 ** -24)
            band = 2.0 * 2 ** -24 * (8 + 4 * np.abs(np.log2(rec[:, 5])) + 4 * np.abs(l64) + 35 * Q + posb)
            r = np.abs(l32.astype(np.float64) - l64)[near] / band[near]
            worst = max(worst, float(r.max(initial=0.0)))
    assert worst <= 1.0, worst


def _fake_gpu_from_outcomes(ref, pick):
    """A "GPU" window built from the oracle's outcomes: for each fragile pixel, outcome pick(p, outcomes)."""
    img = ref["image"].astype(np.float32).copy()
    od = ref["overdraw"].copy()
    rows = ref["alt"]["fwd"]
    w = img.shape[1]
    for p in np.unique(rows["pix"]):
        sel = np.flatnonzero(rows["pix"] == p)
        o = pick(p, rows["outcome"][sel])
        r = sel[list(rows["outcome"][sel]).index(o)]
        y, x = divmod(int(p), w)
        img[y, x] = rows["image"][r]
        od[y, x] = rows["overdraw"][r]
    return img, od


def test_parity_helper_accepts_every_outcome_and_rejects_planted_mistakes():
    sc, cam = synth.tiny_scene(0), synth.tiny_camera()
    g = synth.upstream_gradient(128, 128, seed=4).astype(np.float64)
    ref = oracle.render(sc, cam, "sub", nthreads=4, dl_dimage=g, outcomes=True)
    assert ref["fragile"].any() and not ref["unresolved"].any()
    for pick in (lambda p, o: 0, lambda p, o: int(o.max())):
        img, od = _fake_gpu_from_outcomes(ref, pick)
        m = parity.assert_forward(img, od, ref)
        if pick(0, np.array([0, 1])) == 1:
            assert m.n_alternative > 0
    # a planted mistake: one non-fragile pixel off by 2e-4, one fragile pixel off by one in overdraw
    img, od = _fake_gpu_from_outcomes(ref, lambda p, o: 0)
    y, x = np.argwhere(~ref["fragile"] & (ref["overdraw"] > 0))[0]
    img[y, x, 1] += 2e-4
    yf, xf = np.argwhere(ref["fragile"])[0]
    od[yf, xf] += 1
    m = parity.match_forward(img, od, ref)
    assert {(f[0], f[1]) for f in m.failures} == {(y, x), (yf, xf)}


def test_parity_helper_gradients_follow_the_chosen_outcomes():
    """The reference for pixels that took another outcome equals the oracle's own gradient over a window
    in which those pixels' walk went the other way: checked on a list-level construction. Here: the
    gradient assembled for the all-FP64 choice is the oracle's gradient itself, and a planted 1 % error
    in one element is caught."""
    sc, cam = synth.tiny_scene(0), synth.tiny_camera()
    g = synth.upstream_gradient(128, 128, seed=4).astype(np.float64)
    ref = oracle.render(sc, cam, "lin", nthreads=4, dl_dimage=g, outcomes=True)
    img, od = _fake_gpu_from_outcomes(ref, lambda p, o: 0)
    m = parity.assert_forward(img, od, ref)
    gref = parity.reference_gradients(ref, m)
    for k in parity.PARAM_KEYS:
        assert np.array_equal(gref.d[k], ref["d_" + k].reshape(len(ref["d_means"]), -1))
    fake = {k: ref["d_" + k].copy() for k in parity.PARAM_KEYS}
    rep = parity.compare_gradients(fake, gref)
    assert rep.failed == 0 and rep.scaled == 0
    i = int(np.argmax(np.abs(fake["opacity_logits"])))
    fake["opacity_logits"][i] *= 1.01
    rep = parity.compare_gradients(fake, gref)
    assert rep.failed == 1
