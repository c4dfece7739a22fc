"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function that
include/ngs.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ngs.h")).read()
    return sorted(set(re.findall(r"NGS_API\s+[\w\s\*]+?\b(ngs_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ngs_create", "ngs_destroy", "ngs_render", "ngs_render_backward", "ngs_last_error",
                 "ngs_frame_create", "ngs_frame_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2603_02887_gb300 import _abi, build

    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(_abi.SIGNATURES), "binding and header disagree"
    _abi.load()


def test_default_options_without_gpu():
    from paper_2603_02887_gb300 import _abi

    o = _abi.Options()
    _abi.load().ngs_default_options(ctypes.byref(o))
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    assert (o.tile_w, o.tile_h, o.max_splats) == (16, 16, 0)


def test_built_for_sm103a_only():
    from paper_2603_02887_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_codes_map_to_exceptions_without_gpu():
    import pytest

    from paper_2603_02887_gb300 import _abi

    _abi.check(_abi.NGS_OK, None)
    with pytest.raises(_abi.CapacityExceeded) as e:
        _abi.check(_abi.NGS_ERR_CAPACITY, None)
    assert e.value.code == _abi.NGS_ERR_CAPACITY and isinstance(e.value, _abi.NGSError)
    with pytest.raises(_abi.NGSError) as e:
        _abi.check(_abi.NGS_ERR_DEVICE_CHECK, None)
    assert not isinstance(e.value, _abi.CapacityExceeded)
    # frame entry points refuse a null frame without touching the device
    lib = _abi.load()
    assert lib.ngs_frame_set_async(None, 1) == _abi.NGS_ERR_INVALID_ARG
    assert lib.ngs_frame_status(None, None) == _abi.NGS_ERR_INVALID_ARG


def test_binding_constants_match_the_header():
    from paper_2603_02887_gb300 import _abi

    text = open(os.path.join(ROOT, "include", "ngs.h")).read()
    defines = dict(re.findall(r"#define\s+(NGS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    shared = [k for k in defines if hasattr(_abi, k)]
    assert {"NGS_OK", "NGS_ERR_CAPACITY", "NGS_MODEL_EXP", "NGS_MODEL_QUAD"} <= set(shared)
    for k in shared:
        assert getattr(_abi, k) == int(defines[k]), k
