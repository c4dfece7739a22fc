"""Parity of GPU renders and gradients against the FP64 oracle, checking every pixel.

The oracle takes every compositing decision in FP64 and, where the FP64 value lies within the error bound
of the GPU's FP32 computation of it, enumerates both ways (``oracle.render(..., outcomes=True)``). A GPU
pixel passes when it equals one of its pixel's outcomes: image within ``PIX_TOL`` (max abs), overdraw
exact. Pixels with a single outcome are compared with it directly.

Gradients are sums over pixels, so the reference is assembled from the outcome each pixel took: the
oracle's FP64 gradient (outcome 0 everywhere) plus, for every pixel whose GPU result matched another
outcome, that outcome's record-gradient terms minus outcome 0's, chained to the raw parameters with the
oracle's Jacobians. When a pixel's GPU result matches several outcomes (for example an alpha_max clamp
that changes alpha by less than the image tolerance), the gradient may follow any of them; the sum of
their differences, chained through the absolute Jacobian, is the element's ``allowance``. A colour
channel at its max(0, .) clamp (per Gaussian, not per pixel) may be clamped or not: each combination of
its borderline channels is a candidate reference for that Gaussian's gradients.

The gradient criterion per element (relative 1e-3, with a floor of 1e-3 x the tensor's largest gradient):
  strict:  |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|) + allowance
  scaled:  the same + 1e-4 s + p. A gradient is a sum of per-pixel terms that may cancel; in FP32 it is
           only as accurate as its terms: s (the oracle's sum of the absolute terms chained through the
           absolute Jacobian) bounds the accumulation (a sum of N < 1600 terms in any order moves by at most
           N u s) and the replay's differences of O(1) running sums (1 - S, L0 - sum E pbar, A - E_k taubar_k;
           ~n u), and p (the same sum with each term weighted by the oracle's bound of the relative FP32
           error of its pbar, from the FP32 records and running sums) bounds what the inputs put in.
Every element must pass the scaled criterion; ``GradReport`` counts how many needed the scale terms, which
tests bound.

Test infrastructure only (numpy); it imports nothing from the CUDA path.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

PIX_TOL = 1e-4
GRAD_REL = 1e-3
FLOOR_REL = 1e-3
SCALE_REL = 1e-4
PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@dataclasses.dataclass
class ForwardMatch:
    n_pixels: int
    n_fragile: int        # pixels with more than one outcome
    n_unresolved: int     # pixels whose enumeration was cut short
    n_alternative: int    # pixels whose GPU result matched an outcome other than the FP64 walk
    n_ambiguous: int      # pixels whose GPU result matched several outcomes
    failures: list        # (y, x, reason)
    chosen: dict          # window pixel -> chosen outcome (fragile pixels only)
    others: dict          # window pixel -> other matching outcomes

    def summary(self):
        return (f"{self.n_pixels} px, fragile {self.n_fragile} ({self.n_fragile / max(self.n_pixels, 1):.3%}), "
                f"other outcome {self.n_alternative}, ambiguous {self.n_ambiguous}, unresolved {self.n_unresolved}")


def match_forward(image, overdraw, ref, tol=PIX_TOL):
    """Match a GPU window (image [h, w, 3], overdraw [h, w] or None) to the oracle's outcomes."""
    img = np.asarray(image, np.float64)
    h, w = img.shape[:2]
    frag = ref["fragile"]
    fails = []
    err = np.abs(img - ref["image"]).max(axis=-1)
    ok = err <= tol
    if overdraw is not None:
        ok &= np.asarray(overdraw) == ref["overdraw"]
    for y, x in zip(*np.nonzero(~ok & ~frag)):
        fails.append((int(y), int(x), f"gpu {img[y, x]} od {None if overdraw is None else int(overdraw[y, x])} "
                                      f"vs oracle {ref['image'][y, x]} od {int(ref['overdraw'][y, x])}"))
    chosen, others = {}, {}
    n_alt = n_amb = 0
    alt = ref.get("alt")
    if frag.any():
        assert alt is not None, "fragile pixels need oracle.render(..., outcomes=True)"
        rows = alt["fwd"]
        order = np.argsort(rows["pix"], kind="stable")
        pix_sorted = rows["pix"][order]
        for p in np.flatnonzero(frag.reshape(-1)):
            lo, hi = np.searchsorted(pix_sorted, [p, p + 1])
            y, x = divmod(int(p), w)
            cand = order[lo:hi]
            e = np.abs(rows["image"][cand] - img[y, x]).max(axis=-1)
            m = e <= tol
            if overdraw is not None:
                m &= rows["overdraw"][cand] == overdraw[y, x]
            if not m.any():
                fails.append((y, x, f"gpu {img[y, x]} od {None if overdraw is None else int(overdraw[y, x])} "
                                    f"matches none of {len(cand)} outcomes "
                                    f"{[(int(rows['overdraw'][c]), rows['image'][c].round(6).tolist()) for c in cand]}"))
                continue
            best = cand[m][np.argmin(e[m])]
            chosen[int(p)] = int(rows["outcome"][best])
            others[int(p)] = [int(rows["outcome"][c]) for c in cand[m] if c != best]
            n_alt += chosen[int(p)] != 0
            n_amb += len(others[int(p)]) > 0
    return ForwardMatch(h * w, int(frag.sum()), int(ref["unresolved"].sum()), n_alt, n_amb, fails, chosen, others)


def assert_forward(image, overdraw, ref, tol=PIX_TOL, label=""):
    m = match_forward(image, overdraw, ref, tol)
    assert not m.failures, f"{label}: {len(m.failures)} pixels fail ({m.summary()}): {m.failures[:4]}"
    return m


def _param_layout(K):
    """Slices of the oracle's raw-parameter vector (11 + 3 K) per parameter array."""
    return {"means": slice(0, 3), "log_scales": slice(3, 6), "quats": slice(6, 10), "opacity_logits": slice(10, 11),
            "sh": slice(11, 11 + 3 * K)}


@dataclasses.dataclass
class GradRef:
    d: dict        # reference gradient per parameter array
    s: dict        # error scale
    allow: dict    # outcome-ambiguity allowance
    p: dict        # FP32 input-error scale
    eflip: list    # (gid, [(subset, {key: delta vector [np]})]) candidate adjustments per Gaussian
    layout: dict


def reference_gradients(ref, match: ForwardMatch):
    """The oracle gradient for the outcomes the GPU took (see the module docstring)."""
    n = ref["d_means"].shape[0]
    K = ref["d_sh"].reshape(n, -1, 3).shape[1]
    lay = _param_layout(K)
    d = {k: ref["d_" + k].reshape(n, -1).copy() for k in PARAM_KEYS}
    s = {k: ref["s_" + k].reshape(n, -1).copy() for k in PARAM_KEYS}
    pe = {k: ref["p_" + k].reshape(n, -1).copy() for k in PARAM_KEYS}
    allow = {k: np.zeros_like(d[k]) for k in PARAM_KEYS}
    alt = ref.get("alt")
    delta_rec = None
    if alt is not None and len(alt["grad"]["pix"]):
        g = alt["grad"]
        nj = len(alt["jac_gid"])
        ch_of = np.full(int(g["pix"].max()) + 1, -1, np.int64)
        for p, c in match.chosen.items():
            if p < len(ch_of):
                ch_of[p] = c
        rowc = ch_of[g["pix"]]
        delta_rec = np.zeros((nj, 9))
        abs_rec = np.zeros((nj, 9))
        err_rec = np.zeros((nj, 9))
        amb_rec = np.zeros((nj, 9))
        take = (rowc > 0) & (g["outcome"] == rowc)
        drop = (rowc > 0) & (g["outcome"] == 0)
        np.add.at(delta_rec, g["ju"][take], g["rec"][take, :9])
        np.add.at(delta_rec, g["ju"][drop], -g["rec"][drop, :9])
        np.add.at(abs_rec, g["ju"][take], g["rec"][take, 9:18])
        np.add.at(err_rec, g["ju"][take], g["rec"][take, 18:27])
        for p, oth in match.others.items():
            if not oth:
                continue
            at_p = g["pix"] == p
            tot = {}
            for o in [match.chosen[p]] + oth:
                sel = at_p & (g["outcome"] == o)
                acc = np.zeros((nj, 9))
                np.add.at(acc, g["ju"][sel], g["rec"][sel, :9])
                tot[o] = acc
            for o in oth:
                amb_rec += np.abs(tot[o] - tot[match.chosen[p]])
        J = alt["jac"]
        gid = alt["jac_gid"]
        pd = np.einsum("jr,jrp->jp", delta_rec, J)
        ps = np.einsum("jr,jrp->jp", abs_rec, np.abs(J))
        pp = np.einsum("jr,jrp->jp", err_rec, np.abs(J))
        pa = np.einsum("jr,jrp->jp", amb_rec, np.abs(J))
        for k in PARAM_KEYS:
            np.add.at(d[k], gid, pd[:, lay[k]])
            np.add.at(s[k], gid, ps[:, lay[k]])
            np.add.at(pe[k], gid, pp[:, lay[k]])
            np.add.at(allow[k], gid, pa[:, lay[k]])
    eflip = []
    if alt is not None:
        e = alt["eflip"]
        ju_of = {int(x): i for i, x in enumerate(alt["jac_gid"])} if delta_rec is not None else {}
        for i, gi in enumerate(e["gid"]):
            gE = e["gE"][i].copy()
            if int(gi) in ju_of:
                gE += delta_rec[ju_of[int(gi)], 6:9]
            chans = [c for c in range(3) if (int(e["mask"][i]) >> c) & 1]
            cands = []
            for r in range(len(chans) + 1):
                for sub in itertools.combinations(chans, r):
                    vec = sum((gE[c] * e["dJ"][i, c] for c in sub), np.zeros(e["dJ"].shape[-1]))
                    cands.append((sub, {k: vec[lay[k]] for k in PARAM_KEYS}))
            eflip.append((int(gi), cands))
    return GradRef(d, s, allow, pe, eflip, lay)


def sum_refs(refs):
    """The reference of a sum of renders (for example the views of a batch): gradients, scales and
    allowances add; a Gaussian with borderline colour clamps in several views takes every combination of
    its per-view candidates."""
    out = GradRef({k: sum(r.d[k] for r in refs) for k in PARAM_KEYS},
                  {k: sum(r.s[k] for r in refs) for k in PARAM_KEYS},
                  {k: sum(r.allow[k] for r in refs) for k in PARAM_KEYS},
                  {k: sum(r.p[k] for r in refs) for k in PARAM_KEYS}, [], refs[0].layout)
    by_gid = {}
    for r in refs:
        for gi, cands in r.eflip:
            by_gid.setdefault(gi, []).append(cands)
    for gi, lists in by_gid.items():
        merged = []
        for combo in itertools.product(*lists):
            vec = {k: sum(c[1][k] for c in combo) for k in PARAM_KEYS}
            merged.append((tuple(ch for c in combo for ch in c[0]), vec))
        out.eflip.append((gi, merged))
    return out


@dataclasses.dataclass
class GradReport:
    n: int = 0             # elements compared
    strict: int = 0        # passing without the error-scale term
    scaled: int = 0        # passing only with it
    failed: int = 0
    allowed: int = 0       # elements with a nonzero outcome-ambiguity allowance
    eflip_alt: int = 0     # Gaussians whose colour clamp went the other way
    worst_scaled: float = 0.0  # largest (|g - g_ref| - strict) / (1e-4 s + p) among the scaled ones
    details: list = dataclasses.field(default_factory=list)

    def summary(self):
        return (f"{self.n} elements: strict {self.strict}, needed the scale terms {self.scaled} "
                f"({self.scaled / max(self.n, 1):.3%}), failed {self.failed}; ambiguity allowance on {self.allowed}; "
                f"colour clamps flipped {self.eflip_alt}")


def _tolerances(ref, s, allow, p):
    floor = FLOOR_REL * np.abs(ref).max() if ref.size else 0.0
    strict = GRAD_REL * np.maximum(np.abs(ref), floor) + allow
    return strict, strict + SCALE_REL * s + p


def compare_gradients(gpu, gref: GradRef, exclude=None):
    """Compare GPU gradients (dict key or 'd_'+key -> array) with the reference; returns a GradReport.
    exclude: optional boolean [n] of Gaussians not to compare (none by default)."""
    rep = GradReport()
    n = gref.d["means"].shape[0]
    A = {}
    for k in PARAM_KEYS:
        v = gpu.get(k, gpu.get("d_" + k))
        A[k] = np.asarray(v, np.float64).reshape(n, -1)
    # colour clamps: per Gaussian the candidate adjustment that fits best
    ref = {k: gref.d[k].copy() for k in PARAM_KEYS}
    for gi, cands in gref.eflip:
        best, best_viol = None, None
        for sub, vec in cands:
            viol = 0.0
            for k in PARAM_KEYS:
                r = gref.d[k][gi] + vec[k]
                floor = FLOOR_REL * np.abs(gref.d[k]).max()
                tol = (GRAD_REL * np.maximum(np.abs(r), floor) + gref.allow[k][gi] + SCALE_REL * gref.s[k][gi]
                       + gref.p[k][gi])
                viol = max(viol, float(np.max(np.abs(A[k][gi] - r) / np.maximum(tol, 1e-300))))
            if best_viol is None or viol < best_viol:
                best, best_viol = (sub, vec), viol
        if best[0]:
            rep.eflip_alt += 1
            for k in PARAM_KEYS:
                ref[k][gi] = gref.d[k][gi] + best[1][k]
    for k in PARAM_KEYS:
        a, r, s, al = A[k], ref[k], gref.s[k], gref.allow[k]
        strict, scaled = _tolerances(r, s, al, gref.p[k])
        err = np.abs(a - r)
        keep = np.ones(a.shape, bool) if exclude is None else ~np.asarray(exclude, bool)[:, None].repeat(a.shape[1], 1)
        st = (err <= strict) & keep
        sc = (err <= scaled) & ~st & keep
        bad = (err > scaled) & keep
        rep.n += int(keep.sum())
        rep.strict += int(st.sum())
        rep.scaled += int(sc.sum())
        rep.failed += int(bad.sum())
        rep.allowed += int(((al > 0) & keep).sum())
        if sc.any():
            rep.worst_scaled = max(rep.worst_scaled, float(np.max((err[sc] - strict[sc]) / (scaled[sc] - strict[sc]))))
        for gi, j in list(zip(*np.nonzero(bad)))[:3]:
            rep.details.append(f"{k}[{gi},{j}] gpu={a[gi, j]:.6g} ref={r[gi, j]:.6g} s={s[gi, j]:.3g} "
                               f"p={gref.p[k][gi, j]:.3g} allow={al[gi, j]:.3g}")
    return rep


def assert_gradients(gpu, ref, match, label="", max_scaled=1e-3, exclude=None):
    """Every element within the scaled criterion; at most ``max_scaled`` of them needing the scale term.
    ``ref``/``match`` may be an oracle result and its ForwardMatch, or a GradRef (match None)."""
    gref = ref if isinstance(ref, GradRef) else reference_gradients(ref, match)
    rep = compare_gradients(gpu, gref, exclude=exclude)
    assert rep.failed == 0, f"{label}: {rep.summary()}: {rep.details}"
    assert rep.scaled <= max_scaled * rep.n, f"{label}: {rep.summary()}"
    return rep
