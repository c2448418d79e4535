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


def test_noalloc_rejects_overlapping_user_weights_and_output_without_touching_the_gpu(lib):
    """In user mode the no-alloc kernel reads user_D while it writes D_out: the C entry point
    refuses overlapping ranges before any CUDA call (the pointers are never dereferenced)."""
    from paper_1910_10908_gb300 import _abi
    lib = _abi.load()
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    o.mode = _abi.WEIGHT_MODES["user"]
    base = 0x7f0000000000
    for off in (0, 4 * 100, -4 * 999):               # same array, partial overlaps either way
        o.user_D = base
        assert lib.tffr_weights_noalloc(1000, None, None, 64, 64, ctypes.byref(o), ctypes.c_void_p(base + off),
                                        None, None) == _abi.TFFR_ERR_INVALID_ARG


def test_noalloc_wrapper_checks_lengths_and_devices_before_the_call(monkeypatch):
    """The binding refuses inputs shorter than D_out, and tensors off the current device,
    before it reaches the library (CPU tensors here; the library is never called)."""
    import torch

    import paper_1910_10908_gb300 as tf

    def no_call():
        raise AssertionError("the library must not be reached")

    monkeypatch.setattr(tf._abi, "load", no_call)
    D = torch.empty(100, dtype=torch.float32)
    long_x = torch.zeros(100, dtype=torch.float64)
    short = torch.zeros(99, dtype=torch.float64)
    with pytest.raises(ValueError, match="lam_x"):
        tf.tffr_weights_noalloc(short, long_x, 64, 64, D)
    with pytest.raises(ValueError, match="lam_y"):
        tf.tffr_weights_noalloc(long_x, short, 64, 64, D, separable=True)
    with pytest.raises(ValueError, match="user_D"):
        tf.tffr_weights_noalloc(long_x, long_x, 64, 64, D, mode="user", user_D=torch.zeros(50))
    with pytest.raises(ValueError, match="user_D"):
        tf.tffr_weights_noalloc(long_x, long_x, 64, 64, D, mode="user")
    # a short lam_y is fine when it is not read (range-only weights)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    with pytest.raises(ValueError, match="current CUDA device"):
        tf.tffr_weights_noalloc(long_x, short, 64, 64, D)
