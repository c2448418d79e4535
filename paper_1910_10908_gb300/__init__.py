"""GB300 tFFR: the weighted adjoint NUFFT of thresholded Fourier-frame
reconstruction for stripmap SAR (McKay, Gelb, Jayasuriya, Monga,
arXiv 1910.10908), and its forward twin, as hand-written sm_103a CUDA behind a
C ABI (include/tffr.h).

This module only marshals arguments: torch tensors supply device memory and
the current CUDA stream, every step runs in the library's kernels.  The
functions carry the C names (``tffr_plan``, ``tffr_set_points``,
``tffr_weights``, ``tffr_adjoint``, ``tffr_forward``, ``tffr_destroy``);
``Plan`` wraps them.
"""

from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import VALUES, LAYOUTS, ORDERS, WEIGHT_MODES

__all__ = ["TffrError", "Plan", "tffr_plan", "tffr_set_points", "tffr_weights", "tffr_adjoint",
           "tffr_forward", "tffr_destroy", "tffr_plan_get_info", "tffr_profile", "tffr_profile_read",
           "tffr_weights_noalloc",
           "load_library"]


class TffrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("tffr status %d (%s): %s" % (status, _status_text(status), msg))
        self.status = status


def load_library():
    return _abi.load()


def _status_text(s: int) -> str:
    try:
        return _abi.load().tffr_error_string(int(s)).decode()
    except Exception:  # pragma: no cover
        return "?"


def _check(status: int, plan=None):
    if status != _abi.TFFR_OK:
        msg = ""
        if plan is not None:
            raw = _abi.load().tffr_last_error(plan)
            msg = raw.decode() if raw else ""
        raise TffrError(status, msg)


def _dev(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


# ---- the C entry points, one to one ----

def tffr_plan(Mx: int, My: int, *, width: int = 6, beta: float = 0.0, values: str = "c64",
              layout: str = "auto", order: str = "auto", stream=None) -> ctypes.c_void_p:
    lib = _abi.load()
    o = _abi.tffr_opts()
    lib.tffr_default_opts(ctypes.byref(o))
    o.width = int(width)
    o.beta = float(beta)
    o.values = VALUES[values]
    o.layout = LAYOUTS[layout]
    o.order = ORDERS[order]
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = ctypes.c_void_p()
    _check(lib.tffr_plan(ctypes.byref(handle), int(Mx), int(My), ctypes.byref(o),
                         ctypes.c_void_p(stream.cuda_stream)))
    return handle


def tffr_set_points(plan, lam_x: torch.Tensor, lam_y: torch.Tensor):
    """The library keeps the coordinate pointers: the tensors must outlive their use by the plan."""
    if lam_x.shape != lam_y.shape or lam_x.dim() != 1:
        raise ValueError("lam_x and lam_y must be 1-D of equal length")
    N = lam_x.shape[0]
    px = _dev(lam_x, "lam_x", torch.float64) if N else None
    py = _dev(lam_y, "lam_y", torch.float64) if N else None
    _check(_abi.load().tffr_set_points(plan, N, px, py), plan)


def tffr_weights(plan, *, mode: str = "tffr", separable: bool = False, a: float = 0.01, q: float = 3.0,
                 tau: float = 0.97, user_D: torch.Tensor | None = None, D_out: torch.Tensor | None = None,
                 count: bool = True):
    lib = _abi.load()
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    o.mode = WEIGHT_MODES[mode]
    o.separable = 1 if separable else 0
    o.a, o.q, o.tau = float(a), float(q), float(tau)
    if user_D is not None:
        o.user_D = _dev(user_D, "user_D", torch.float32).value
    pd = _dev(D_out, "D_out", torch.float32) if D_out is not None and D_out.numel() else None
    kept = ctypes.c_int64(-1)
    _check(lib.tffr_weights(plan, ctypes.byref(o), pd, ctypes.byref(kept) if count else None), plan)
    return int(kept.value) if count else None


def tffr_adjoint(plan, values: torch.Tensor, image: torch.Tensor):
    pv = _dev(values, "values") if values.numel() else None
    _check(_abi.load().tffr_adjoint(plan, pv, _dev(image, "image", torch.complex64)), plan)


def tffr_forward(plan, image: torch.Tensor, values: torch.Tensor, apply_weights: bool = True):
    pv = _dev(values, "values") if values.numel() else None
    _check(_abi.load().tffr_forward(plan, _dev(image, "image", torch.complex64), pv, 1 if apply_weights else 0),
           plan)


def tffr_normal_setup(plan):
    _check(_abi.load().tffr_normal_setup(plan), plan)


def tffr_normal_apply(plan, image_in: torch.Tensor, image_out: torch.Tensor):
    _check(_abi.load().tffr_normal_apply(plan, _dev(image_in, "image_in", torch.complex64),
                                         _dev(image_out, "image_out", torch.complex64)), plan)


def tffr_weights_noalloc(lam_x: torch.Tensor, lam_y: torch.Tensor, Mx: int, My: int, D_out: torch.Tensor, *,
                         mode: str = "tffr", separable: bool = False, a: float = 0.01, q: float = 3.0,
                         tau: float = 0.97, user_D: torch.Tensor | None = None, count: bool = True, stream=None):
    """Weights without a plan and without device allocation (see include/tffr.h)."""
    lib = _abi.load()
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    o.mode = WEIGHT_MODES[mode]
    o.separable = 1 if separable else 0
    o.a, o.q, o.tau = float(a), float(q), float(tau)
    if user_D is not None:
        o.user_D = _dev(user_D, "user_D", torch.float32).value
    N = int(D_out.shape[0])
    px = _dev(lam_x, "lam_x", torch.float64) if N else None
    py = _dev(lam_y, "lam_y", torch.float64) if N else None
    pd = _dev(D_out, "D_out", torch.float32) if N else None
    if stream is None:
        stream = torch.cuda.current_stream()
    kept = ctypes.c_int64(-1)
    _check(lib.tffr_weights_noalloc(N, px, py, int(Mx), int(My), ctypes.byref(o), pd,
                                    ctypes.byref(kept) if count else None, ctypes.c_void_p(stream.cuda_stream)))
    return int(kept.value) if count else None


def tffr_plan_get_info(plan) -> dict:
    info = _abi.tffr_plan_info()
    _check(_abi.load().tffr_plan_get_info(plan, ctypes.byref(info)), plan)
    return {name: getattr(info, name) for name, _ in info._fields_}


def tffr_profile(plan, enable: bool):
    _check(_abi.load().tffr_profile(plan, 1 if enable else 0), plan)


def tffr_profile_read(plan) -> dict:
    n = len(_abi.STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(_abi.load().tffr_profile_read(plan, ms, cnt, n), plan)
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(_abi.STAGES)}


def tffr_destroy(plan):
    _check(_abi.load().tffr_destroy(plan))


# ---- convenience wrapper ----

_VALUE_DTYPES = {"c64": (torch.complex64,), "c128": (torch.complex128,), "f16": (torch.complex32,),
                 "bf16": (torch.bfloat16,)}


class Plan:
    """One image size, one point set, one set of weights; adjoint and forward on demand."""

    def __init__(self, Mx: int, My: int | None = None, *, width: int = 6, beta: float = 0.0,
                 values: str = "c64", layout: str = "auto", order: str = "auto", device=None):
        self.Mx, self.My = int(Mx), int(My if My is not None else Mx)
        self.values = values
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream()
            self._h = tffr_plan(self.Mx, self.My, width=width, beta=beta, values=values, layout=layout,
                                order=order, stream=self.stream)
        self.N = None          # samples of the last set_points (None before)

    def _handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def set_points(self, lam_x: torch.Tensor, lam_y: torch.Tensor) -> "Plan":
        """The plan reads the coordinate tensors in place: keep references to them."""
        tffr_set_points(self._handle(), lam_x, lam_y)
        self._coords = (lam_x, lam_y)
        self.N = int(lam_x.shape[0])
        return self

    def weights(self, **kw):
        return tffr_weights(self._handle(), **kw)

    def value_tensor(self, n: int | None = None) -> torch.Tensor:
        n = (self.N or 0) if n is None else n
        if self.values == "bf16":
            return torch.empty((n, 2), dtype=torch.bfloat16, device=self.device)
        return torch.empty(n, dtype=_VALUE_DTYPES[self.values][0], device=self.device)

    def adjoint(self, values: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if values.dtype not in _VALUE_DTYPES[self.values]:
            raise TypeError("values dtype %s does not match the plan's %s" % (values.dtype, self.values))
        if self.N is not None and values.shape[0] != self.N:
            raise ValueError("expected %d samples, got %d" % (self.N, values.shape[0]))
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        tffr_adjoint(self._handle(), values, out)
        return out

    def forward(self, image: torch.Tensor, out: torch.Tensor | None = None,
                apply_weights: bool = True) -> torch.Tensor:
        if tuple(image.shape) != (self.My, self.Mx):
            raise ValueError("image must be [My, Mx] = [%d, %d]" % (self.My, self.Mx))
        if out is None:
            dt = torch.complex128 if self.values == "c128" else torch.complex64
            out = torch.empty(self.N or 0, dtype=dt, device=self.device)
        tffr_forward(self._handle(), image, out, apply_weights)
        return out

    def normal_setup(self) -> "Plan":
        """Build the Toeplitz normal operator E^H D E for the current points and weights."""
        tffr_normal_setup(self._handle())
        return self

    def normal(self, image: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """E^H D E image (after normal_setup)."""
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        tffr_normal_apply(self._handle(), image, out)
        return out

    def info(self) -> dict:
        return tffr_plan_get_info(self._handle())

    def profile(self, enable: bool = True):
        tffr_profile(self._handle(), enable)

    def profile_read(self) -> dict:
        """Per stage: (summed milliseconds, timed executions) since profile(True)."""
        return tffr_profile_read(self._handle())

    def close(self):
        if getattr(self, "_h", None) is not None:
            tffr_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
