"""FP64 CPU oracle for generalized non-exponential Gaussian splatting.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path, and the product path
never routes through it.

The arithmetic lives in ``ngs_oracle.c`` (plain C, FP64, one pthread per row band); this module only
marshals numpy arrays through ctypes. What each C function computes and which passage of the paper it
follows is stated in the C file's header:

* ``composite_list`` -- the compositing operator over one ordered list (Sec. 4.2, Eq. generalized_gaussian,
  Eq. nexp_p, Table 1) and its adjoint (App. C for the quadratic family).
* ``project`` / ``project_jacobian`` -- EWA projection of 3D Gaussians to splat records (Sec. 3 baseline).
* ``render`` -- per-pixel rendering with no tiles, optionally with the gradient w.r.t. the raw parameters.

Options are rounded to FP32 before they reach the C code, because the GPU library receives them as
FP32: both sides then compare against the same threshold values.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ngs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libngs_oracle.so")
_lib = None

EXP, QUAD, BLEND, VICINI = 0, 1, 2, 3

#: The four models of the paper's experiments (Sec. 5): exponential, and the quadratic mother
#: transmittance with c = -0.5 (sub-linear), 0 (linear) and +0.5 (super-linear).
MODELS = {"exp": (EXP, 0.0), "sub": (QUAD, -0.5), "lin": (QUAD, 0.0), "sup": (QUAD, 0.5)}

DEFAULT_OPTS = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, t_eps=1e-4, dilation=0.3, near_plane=0.2,
                    background=(0.0, 0.0, 0.0), max_splats=0)


def build(force: bool = False) -> str:
    """Compile ngs_oracle.c into _build/libngs_oracle.so (gcc, FP contraction off)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("viewmat", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("param", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_eps", C.c_double),
                ("dilation", C.c_double), ("near_plane", C.c_double), ("background", C.c_double * 3),
                ("max_splats", C.c_int32)]


class _Window(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32), ("h", C.c_int32)]


class _Fwd(C.Structure):
    _fields_ = [("image", C.c_void_p), ("overdraw", C.c_void_p), ("n_listed", C.c_void_p),
                ("fragile", C.c_void_p), ("signature", C.c_void_p), ("n_outcomes", C.c_void_p)]


class _Alt(C.Structure):
    _fields_ = [("n_fwd", C.c_int64), ("fwd_pix", C.c_void_p), ("fwd_outcome", C.c_void_p),
                ("fwd_overdraw", C.c_void_p), ("fwd_image", C.c_void_p),
                ("n_grad", C.c_int64), ("grad_pix", C.c_void_p), ("grad_outcome", C.c_void_p),
                ("grad_ju", C.c_void_p), ("grad_rec", C.c_void_p),
                ("n_params", C.c_int32), ("n_jac", C.c_int64), ("jac_gid", C.c_void_p), ("jac", C.c_void_p),
                ("n_eflip", C.c_int64), ("eflip_gid", C.c_void_p), ("eflip_mask", C.c_void_p),
                ("eflip_dJ", C.c_void_p), ("eflip_gE", C.c_void_p)]


class _Bwd(C.Structure):
    _fields_ = [("dl_dimage", C.c_void_p), ("d_means", C.c_void_p), ("d_log_scales", C.c_void_p),
                ("d_quats", C.c_void_p), ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p),
                ("fragile_gauss", C.c_void_p), ("s_means", C.c_void_p), ("s_log_scales", C.c_void_p),
                ("s_quats", C.c_void_p), ("s_opacity_logits", C.c_void_p), ("s_sh", C.c_void_p),
                ("p_means", C.c_void_p), ("p_log_scales", C.c_void_p), ("p_quats", C.c_void_p),
                ("p_opacity_logits", C.c_void_p), ("p_sh", C.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER
        lib.orc_render.argtypes = [P(_Scene), P(_Camera), P(_Model), P(_Opts), P(_Window), C.c_int, C.c_int,
                                   P(_Fwd), P(_Bwd), P(_Alt)]
        lib.orc_free_alt.argtypes = [P(_Alt)]
        lib.orc_project.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]
        lib.orc_composite_outcomes.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double,
                                               C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_composite_outcomes.restype = C.c_int32
        lib.orc_project_jacobian.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int64, C.c_void_p, C.c_int32]
        lib.orc_composite_list.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_void_p, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_composite_list.restype = C.c_int32
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f32(x):
    return float(np.float32(x))


def _scene(scene, keep):
    means = _f64(scene["means"]).reshape(-1, 3)
    n = means.shape[0]
    ls = _f64(scene["log_scales"]).reshape(n, 3)
    qs = _f64(scene["quats"]).reshape(n, 4)
    op = _f64(scene["opacity_logits"]).reshape(n)
    sh = _f64(scene["sh"]).reshape(n, -1, 3)
    keep += [means, ls, qs, op, sh]
    deg = int(round(np.sqrt(sh.shape[1]))) - 1
    assert (deg + 1) ** 2 == sh.shape[1], "SH coefficient count must be (d+1)^2"
    return _Scene(n, deg, _ptr(means), _ptr(ls), _ptr(qs), _ptr(op), _ptr(sh)), n, sh.shape[1]


def _camera(cam):
    c = _Camera()
    vm = np.asarray(cam["viewmat"], dtype=np.float32).reshape(12).astype(np.float64)
    for i in range(12):
        c.viewmat[i] = vm[i]
    c.fx, c.fy, c.cx, c.cy = (_f32(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def _opts(opts):
    o = dict(DEFAULT_OPTS)
    o.update(opts or {})
    r = _Opts()
    r.alpha_min, r.alpha_max, r.t_eps = _f32(o["alpha_min"]), _f32(o["alpha_max"]), _f32(o["t_eps"])
    r.dilation, r.near_plane = _f32(o["dilation"]), _f32(o["near_plane"])
    for i in range(3):
        r.background[i] = _f32(o["background"][i])
    r.max_splats = int(o["max_splats"])
    return r


def _model(model):
    if isinstance(model, str):
        model = MODELS[model]
    return _Model(int(model[0]), float(model[1]))


def composite_list(alpha, E, model, t_eps=0.0, max_splats=0, background=(0.0, 0.0, 0.0), g=None):
    """The compositing operator over one front-to-back list (no alpha_min filter, no geometry).

    Returns dict(pbar[n], color[3], T_end, m, saturated) and, when ``g`` = dL/dL0 is given,
    dalpha[n] and dE[n, 3]. Entries past the stop have pbar = 0.
    """
    lib = _load()
    alpha = _f64(alpha).reshape(-1)
    n = alpha.shape[0]
    E = _f64(E).reshape(n, 3)
    bg = _f64(background).reshape(3)
    m_ = _model(model)
    pbar = np.zeros(n)
    out4 = np.zeros(4)
    sat = C.c_int32(0)
    gg = None if g is None else _f64(g).reshape(3)
    dal = np.zeros(n) if g is not None else None
    dE = np.zeros((n, 3)) if g is not None else None
    m = lib.orc_composite_list(m_.kind, m_.param, float(t_eps), int(max_splats), _ptr(bg), n, _ptr(alpha), _ptr(E),
                               _ptr(pbar), _ptr(out4), C.byref(sat), _ptr(gg), _ptr(dal), _ptr(dE))
    res = dict(pbar=pbar, color=out4[:3].copy(), T_end=float(out4[3]), m=int(m), saturated=bool(sat.value))
    if g is not None:
        res.update(dalpha=dal, dE=dE)
    return res


def project(scene, camera, opts=None):
    """EWA projection of every Gaussian: rec[n, 10] = (u, v, A, B, C, aleph, E0, E1, E2, rbound), the FP32
    sort depth z32[n], valid[n] (in front of the near plane and able to reach alpha_min), and the error
    bounds the oracle assumes for the GPU's FP32 records: pos_err[n, 2] (pixels) of (u, v) and e_band[n, 3]
    of the colour channels before their max(0, .) clamp."""
    lib = _load()
    keep = []
    sc, n, _ = _scene(scene, keep)
    cam, o = _camera(camera), _opts(opts)
    rec = np.zeros((n, 10))
    z32 = np.zeros(n, dtype=np.float32)
    valid = np.zeros(n, dtype=np.int32)
    pos_err = np.zeros((n, 2))
    e_band = np.zeros((n, 3))
    lib.orc_project(C.byref(sc), C.byref(cam), C.byref(o), _ptr(rec), _ptr(z32), _ptr(valid), _ptr(pos_err),
                    _ptr(e_band))
    return dict(rec=rec, z32=z32, valid=valid.astype(bool), pos_err=pos_err, e_band=e_band)


def composite_outcomes(raw, E, model, band=None, alpha_min=0.0, alpha_max=np.inf, t_eps=0.0, max_splats=0,
                       background=(0.0, 0.0, 0.0), max_out=64):
    """Every outcome of one list's walk when the decisions within ``band`` (log2-domain error bound per
    candidate; None: exact) of their thresholds may go either way. Returns a list of dict(m, color, T_end,
    pbar[n]) (outcome 0 = the FP64 walk), or None when there were more than ``max_out``."""
    lib = _load()
    raw = _f64(raw).reshape(-1)
    n = raw.shape[0]
    E = _f64(E).reshape(n, 3)
    bg = _f64(background).reshape(3)
    b = None if band is None else _f64(np.broadcast_to(band, (n,)))
    m_ = _model(model)
    ms = np.zeros(max_out, np.int32)
    out4 = np.zeros((max_out, 4))
    pbar = np.zeros((max_out, max(n, 1)))
    cnt = lib.orc_composite_outcomes(m_.kind, m_.param, float(alpha_min), float(alpha_max), float(t_eps),
                                     int(max_splats), _ptr(bg), n, _ptr(raw), _ptr(b), _ptr(E), int(max_out),
                                     _ptr(ms), _ptr(out4), _ptr(pbar))
    if cnt < 0:
        return None
    return [dict(m=int(ms[i]), color=out4[i, :3].copy(), T_end=float(out4[i, 3]), pbar=pbar[i, :n].copy())
            for i in range(cnt)]


def project_jacobian(scene, camera, g, opts=None, eflip=0):
    """Jacobian [9, 11 + 3K] of (u, v, A, B, C, aleph, E0, E1, E2) w.r.t. (mean 3, log-scale 3, quat 4,
    opacity logit 1, SH 3K) of Gaussian ``g``, by complex step. Bit ch of ``eflip`` takes colour channel
    ch's max(0, .) clamp against the sign of its value."""
    lib = _load()
    keep = []
    sc, n, K = _scene(scene, keep)
    cam, o = _camera(camera), _opts(opts)
    jac = np.zeros((9, 11 + 3 * K))
    lib.orc_project_jacobian(C.byref(sc), C.byref(cam), C.byref(o), int(g), _ptr(jac), int(eflip))
    return jac


def render(scene, camera, model, opts=None, window=None, nthreads=1, brute_force=False, dl_dimage=None,
           outcomes=False):
    """Render a window (x0, y0, w, h) of ``camera`` (default: the full image) per pixel in FP64.

    Returns dict(image[h, w, 3], overdraw[h, w], n_listed[h, w], fragile[h, w], signature[h, w],
    n_outcomes[h, w]) and, when ``dl_dimage`` [h, w, 3] is given, the gradients d_means, d_log_scales,
    d_quats, d_opacity_logits, d_sh (same shapes as the parameters), fragile_gauss[n] (bit ch: colour
    channel ch is borderline at its max(0, .) clamp) and, per gradient, its error scale s_* (the sum of the
    absolute per-pixel terms chained through the absolute Jacobian) and p_* (the same with each term
    weighted by the bound of the relative FP32 error of its splat's pbar at that pixel). Image, overdraw
    and gradients are
    those of the FP64 walk. ``fragile`` is 1 where a decision of the pixel's walk is borderline (within the
    FP32 error bound of its threshold) and 2 where the enumeration was cut short (``unresolved``).

    With ``outcomes`` the borderline decisions of every pixel are enumerated and ``alt`` holds every
    outcome of every pixel that has more than one: ``fwd`` rows (pix = y w + x in the window, outcome,
    overdraw, image[3]), with ``dl_dimage`` also ``grad`` rows (pix, outcome, ju, rec[27]: the per-entry
    record-gradient terms, their absolute values and their FP32 error bounds), ``jac`` [n_jac, 9, np] with ``jac_gid`` (the
    Jacobians of the Gaussians named by ``ju``), and ``eflip`` (gid, mask, dJ [., 3, np], gE [., 3]) for
    Gaussians with a borderline colour clamp.
    """
    lib = _load()
    keep = []
    sc, n, K = _scene(scene, keep)
    cam, o, m_ = _camera(camera), _opts(opts), _model(model)
    if window is None:
        window = (0, 0, cam.width, cam.height)
    x0, y0, w, h = (int(v) for v in window)
    win = _Window(x0, y0, w, h)
    image = np.zeros((h, w, 3))
    overdraw = np.zeros((h, w), dtype=np.int32)
    n_listed = np.zeros((h, w), dtype=np.int32)
    fragile = np.zeros((h, w), dtype=np.uint8)
    sig = np.zeros((h, w), dtype=np.uint64)
    nout = np.zeros((h, w), dtype=np.int32)
    fwd = _Fwd(_ptr(image), _ptr(overdraw), _ptr(n_listed), _ptr(fragile), _ptr(sig), _ptr(nout))
    res = dict(image=image, overdraw=overdraw, n_listed=n_listed, signature=sig, n_outcomes=nout)
    bwd_p = None
    if dl_dimage is not None:
        dl = _f64(dl_dimage).reshape(h, w, 3)
        grads = dict(d_means=np.zeros((n, 3)), d_log_scales=np.zeros((n, 3)), d_quats=np.zeros((n, 4)),
                     d_opacity_logits=np.zeros(n), d_sh=np.zeros((n, K, 3)))
        fg = np.zeros(n, dtype=np.uint8)
        names = ("means", "log_scales", "quats", "opacity_logits", "sh")
        scales = {"s_" + k: np.zeros_like(grads["d_" + k]) for k in names}
        scales.update({"p_" + k: np.zeros_like(grads["d_" + k]) for k in names})
        grads.update(scales)
        bwd = _Bwd(_ptr(dl), *(_ptr(grads["d_" + k]) for k in names), _ptr(fg),
                   *(_ptr(scales["s_" + k]) for k in names), *(_ptr(scales["p_" + k]) for k in names))
        bwd_p = C.byref(bwd)
        keep.append(dl)
    alt = _Alt() if outcomes else None
    lib.orc_render(C.byref(sc), C.byref(cam), C.byref(m_), C.byref(o), C.byref(win), int(nthreads),
                   int(bool(brute_force)), C.byref(fwd), bwd_p, C.byref(alt) if alt is not None else None)
    res["fragile"] = fragile > 0
    res["unresolved"] = fragile == 2
    if dl_dimage is not None:
        res.update(grads)
        res["fragile_gauss"] = fg
    if alt is not None:
        try:
            res["alt"] = _alt_arrays(alt)
        finally:
            lib.orc_free_alt(C.byref(alt))
    return res


def _copy(ptr, n, dtype, shape=None):
    if n == 0 or not ptr:
        return np.zeros((0,) + tuple(shape or ()), dtype=dtype)
    count = int(n * (np.prod(shape) if shape else 1))
    arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(np.ctypeslib.as_ctypes_type(dtype))), shape=(count,))
    return arr.copy().reshape((n,) + tuple(shape or ()))


def _alt_arrays(a):
    npar = int(a.n_params)
    return dict(
        fwd=dict(pix=_copy(a.fwd_pix, a.n_fwd, np.int64), outcome=_copy(a.fwd_outcome, a.n_fwd, np.int32),
                 overdraw=_copy(a.fwd_overdraw, a.n_fwd, np.int32), image=_copy(a.fwd_image, a.n_fwd, np.float64, (3,))),
        grad=dict(pix=_copy(a.grad_pix, a.n_grad, np.int64), outcome=_copy(a.grad_outcome, a.n_grad, np.int32),
                  ju=_copy(a.grad_ju, a.n_grad, np.int32), rec=_copy(a.grad_rec, a.n_grad, np.float64, (27,))),
        jac=_copy(a.jac, a.n_jac, np.float64, (9, npar)), jac_gid=_copy(a.jac_gid, a.n_jac, np.int64),
        eflip=dict(gid=_copy(a.eflip_gid, a.n_eflip, np.int64), mask=_copy(a.eflip_mask, a.n_eflip, np.uint8),
                   dJ=_copy(a.eflip_dJ, a.n_eflip, np.float64, (3, npar)),
                   gE=_copy(a.eflip_gE, a.n_eflip, np.float64, (3,))),
    )
