"""ctypes view of the C ABI in include/tffr.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_tffr.so")

TFFR_OK = 0
TFFR_ERR_INVALID_ARG = 1
TFFR_ERR_NOT_READY = 2
TFFR_ERR_CUDA = 3
TFFR_ERR_OOM = 4
TFFR_ERR_TIMEOUT = 5

VALUES = {"c64": 0, "c128": 1, "f16": 2, "bf16": 3}
LAYOUTS = {"auto": 0, "general": 1, "rows": 2}
ORDERS = {"auto": 0, "fine_rows": 1}
WEIGHT_MODES = {"tffr": 0, "unit": 1, "user": 2}


class tffr_opts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_int), ("width", ctypes.c_int), ("beta", ctypes.c_double),
                ("values", ctypes.c_int), ("layout", ctypes.c_int), ("order", ctypes.c_int)]


class tffr_weight_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("separable", ctypes.c_int), ("a", ctypes.c_double),
                ("q", ctypes.c_double), ("tau", ctypes.c_double), ("user_D", ctypes.c_void_p)]


class tffr_plan_info(ctypes.Structure):
    _fields_ = [("Mx", ctypes.c_int), ("My", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("width", ctypes.c_int), ("beta", ctypes.c_double), ("N", ctypes.c_int64),
                ("layout", ctypes.c_int), ("n_rows", ctypes.c_int64), ("row_cells", ctypes.c_int64),
                ("max_row_cells", ctypes.c_int), ("n_kept", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_int64), ("pulse_order", ctypes.c_int)]


class tffr_batch_info(ctypes.Structure):
    _fields_ = [("n_patches", ctypes.c_int), ("n_classes", ctypes.c_int), ("samples", ctypes.c_int64),
                ("tuned", ctypes.c_int), ("width", ctypes.c_int), ("spread_ms", ctypes.c_float),
                ("class_side", ctypes.c_int * 8),
                ("class_patches", ctypes.c_int * 8), ("class_blocks", ctypes.c_int * 8),
                ("class_ms", ctypes.c_float * 8)]


STAGES = ["points", "weights", "spread", "row_fft", "col_fft", "fwd_col_fft", "fwd_row_fft", "interp"]


# name -> (restype, argtypes), exactly the declarations of include/tffr.h
SIGNATURES = {
    "tffr_default_opts": (None, [ctypes.POINTER(tffr_opts)]),
    "tffr_default_weight_opts": (None, [ctypes.POINTER(tffr_weight_opts)]),
    "tffr_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(tffr_opts), ctypes.c_void_p]),
    "tffr_set_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tffr_weight_opts), ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_int64)]),
    "tffr_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_reconstruct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(tffr_weight_opts), ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tffr_adjoint_unweighted": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_weight_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_cg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double)]),
    "tffr_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tffr_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "tffr_weights_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(tffr_weight_opts), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "tffr_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "tffr_batch_adjoint": (ctypes.c_int, [ctypes.c_void_p]),
    "tffr_batch_wait": (ctypes.c_int, [ctypes.c_void_p]),
    "tffr_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tffr_batch_set_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "tffr_batch_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tffr_batch_info)]),
    "tffr_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tffr_normal_setup": (ctypes.c_int, [ctypes.c_void_p]),
    "tffr_normal_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tffr_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tffr_plan_info)]),
    "tffr_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tffr_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tffr_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}

_LIB = None


def load():
    """Load the built library; raise if it is missing (there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "the tFFR CUDA library is not built (%s missing); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB
