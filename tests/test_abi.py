"""The C ABI library builds, loads and exports every entry point its header declares (CPU only)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tffr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(tffr_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_10908_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("tffr_plan", "tffr_set_points", "tffr_weights", "tffr_adjoint", "tffr_forward", "tffr_destroy"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_1910_10908_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == declared_functions()


def test_defaults_and_status_strings(lib):
    from paper_1910_10908_gb300 import _abi
    lib = _abi.load()
    o = _abi.tffr_opts()
    lib.tffr_default_opts(ctypes.byref(o))
    assert (o.sigma, o.width, o.beta, o.values, o.layout) == (2, 6, 0.0, 0, 0)
    w = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(w))
    assert (w.mode, w.separable, w.a, w.q, w.tau) == (0, 0, 0.01, 3.0, 0.97)
    assert lib.tffr_error_string(2).decode().startswith("not ready")
    assert lib.tffr_error_string(99).decode() == "unknown status"


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    from paper_1910_10908_gb300 import _abi
    lib = _abi.load()
    assert lib.tffr_plan(None, 64, 64, None, None) == _abi.TFFR_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    # sizes are validated before any CUDA call
    assert lib.tffr_plan(ctypes.byref(h), 48, 64, None, None) == _abi.TFFR_ERR_INVALID_ARG
    assert lib.tffr_plan(ctypes.byref(h), 64, 16384, None, None) == _abi.TFFR_ERR_INVALID_ARG
    o = _abi.tffr_opts()
    lib.tffr_default_opts(ctypes.byref(o))
    o.width = 5
    assert lib.tffr_plan(ctypes.byref(h), 64, 64, ctypes.byref(o), None) == _abi.TFFR_ERR_INVALID_ARG
    assert lib.tffr_set_points(None, 0, None, None) == _abi.TFFR_ERR_INVALID_ARG
    assert lib.tffr_adjoint(None, None, None) == _abi.TFFR_ERR_INVALID_ARG
    assert lib.tffr_destroy(None) == _abi.TFFR_OK
    assert lib.tffr_last_error(None) == b""


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1910_10908_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower().replace("oracle_", ""), f
