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

__all__ = ["TffrError", "Plan", "tffr_plan", "tffr_set_points", "tffr_weights", "tffr_adjoint", "tffr_reconstruct",
           "tffr_forward", "tffr_destroy", "tffr_plan_get_info", "tffr_profile", "tffr_profile_read",
           "tffr_weights_noalloc", "tffr_adjoint_unweighted", "tffr_weight_grad", "tffr_cg",
           "tffr_batch_create", "tffr_batch_adjoint", "tffr_batch_wait", "tffr_batch_tune",
           "tffr_batch_set_wait", "tffr_batch_get_info", "tffr_batch_destroy",
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


def _weight_opts(lib, mode: str, separable: bool, a: float, q: float, tau: float, user_D):
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    o.mode = WEIGHT_MODES[mode]
    o.separable = 1 if separable else 0
    o.a, o.q, o.tau = float(a), float(q), float(tau)
    if user_D is not None:
        o.user_D = _dev(user_D, "user_D", torch.float32).value
    return o


def tffr_weights(plan, *, mode: str = "tffr", separable: bool = False, a: float = 0.01, q: float = 3.0,
                 tau: float = 0.97, user_D: torch.Tensor | None = None, D_out: torch.Tensor | None = None,
                 count: bool = True):
    lib = _abi.load()
    o = _weight_opts(lib, mode, separable, a, q, tau, user_D)
    pd = _dev(D_out, "D_out", torch.float32) if D_out is not None and D_out.numel() else None
    kept = ctypes.c_int64(-1)
    _check(lib.tffr_weights(plan, ctypes.byref(o), pd, ctypes.byref(kept) if count else None), plan)
    return int(kept.value) if count else None


def tffr_adjoint(plan, values: torch.Tensor, image: torch.Tensor):
    pv = _dev(values, "values") if values.numel() else None
    _check(_abi.load().tffr_adjoint(plan, pv, _dev(image, "image", torch.complex64)), plan)


def tffr_reconstruct(plan, lam_x: torch.Tensor, lam_y: torch.Tensor, values: torch.Tensor, image: torch.Tensor, *,
                     mode: str = "tffr", separable: bool = False, a: float = 0.01, q: float = 3.0,
                     tau: float = 0.97, user_D: torch.Tensor | None = None):
    """set_points + weights + adjoint in one library call (the coordinates are kept by pointer)."""
    if lam_x.shape != lam_y.shape or lam_x.dim() != 1:
        raise ValueError("lam_x and lam_y must be 1-D of equal length")
    N = lam_x.shape[0]
    if values.shape[0] != N:
        raise ValueError("values must hold one sample per coordinate")
    if user_D is not None and user_D.numel() < N:
        raise ValueError("user_D shorter than the samples")
    lib = _abi.load()
    o = _weight_opts(lib, mode, separable, a, q, tau, user_D)
    px = _dev(lam_x, "lam_x", torch.float64) if N else None
    py = _dev(lam_y, "lam_y", torch.float64) if N else None
    pv = _dev(values, "values") if values.numel() else None
    _check(lib.tffr_reconstruct(plan, N, px, py, ctypes.byref(o), pv, _dev(image, "image", torch.complex64)), plan)


def tffr_forward(plan, image: torch.Tensor, values: torch.Tensor, apply_weights: bool = True):
    pv = _dev(values, "values") if values.numel() else None
    _check(_abi.load().tffr_forward(plan, _dev(image, "image", torch.complex64), pv, 1 if apply_weights else 0),
           plan)


def tffr_adjoint_unweighted(plan, values: torch.Tensor, image: torch.Tensor):
    pv = _dev(values, "values") if values.numel() else None
    _check(_abi.load().tffr_adjoint_unweighted(plan, pv, _dev(image, "image", torch.complex64)), plan)


def tffr_weight_grad(plan, grad_image: torch.Tensor, values: torch.Tensor, grad_D: torch.Tensor):
    n = values.shape[0]
    pv = _dev(values, "values") if n else None
    pg = _dev(grad_D, "grad_D", torch.float32) if n else None
    _check(_abi.load().tffr_weight_grad(plan, _dev(grad_image, "grad_image", torch.complex64), pv, pg), plan)


def tffr_cg(plan, values: torch.Tensor, image: torch.Tensor, iters: int, use_toeplitz: bool = False,
            residuals: bool = True):
    pv = _dev(values, "values") if values.numel() else None
    hist = (ctypes.c_double * (int(iters) + 1))() if residuals else None
    _check(_abi.load().tffr_cg(plan, pv, _dev(image, "image", torch.complex64), int(iters),
                               1 if use_toeplitz else 0, hist), plan)
    return [float(v) for v in hist] if residuals else None


def tffr_batch_create(plans, values, images, stream=None) -> ctypes.c_void_p:
    """A batch of plans (their handles) with fixed value and image tensors, one per plan."""
    n = len(plans)
    if not (len(values) == len(images) == n) or n == 0:
        raise ValueError("one value tensor and one image per plan")
    hp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h.value) for h in plans])
    hv = (ctypes.c_void_p * n)(*[_dev(v, "values", torch.complex64) for v in values])
    hi = (ctypes.c_void_p * n)(*[_dev(im, "image", torch.complex64) for im in images])
    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_void_p()
    _check(_abi.load().tffr_batch_create(hp, n, hv, hi, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out)))
    return out


def tffr_batch_adjoint(batch):
    _check(_abi.load().tffr_batch_adjoint(batch))


def tffr_batch_wait(batch):
    """Synchronise; raises TffrError (status TIMEOUT) when a wait of an earlier adjoint ran out."""
    _check(_abi.load().tffr_batch_wait(batch))


def tffr_batch_tune(batch, reps: int = 5):
    _check(_abi.load().tffr_batch_tune(batch, int(reps)))


def tffr_batch_set_wait(batch, wait_s: float = 1.0, hold_rows: bool = False):
    _check(_abi.load().tffr_batch_set_wait(batch, float(wait_s), 1 if hold_rows else 0))


def tffr_batch_get_info(batch) -> dict:
    info = _abi.tffr_batch_info()
    _check(_abi.load().tffr_batch_get_info(batch, ctypes.byref(info)))
    k = info.n_classes
    out = {"n_patches": info.n_patches, "n_classes": k, "samples": info.samples, "tuned": bool(info.tuned),
           "width": info.width, "spread_ms": info.spread_ms}
    out["classes"] = [{"side": info.class_side[i], "patches": info.class_patches[i],
                       "blocks": info.class_blocks[i], "ms": info.class_ms[i]} for i in range(min(k, 8))]
    return out


def tffr_batch_destroy(batch):
    _check(_abi.load().tffr_batch_destroy(batch))


def tffr_normal_setup(plan):
    _check(_abi.load().tffr_normal_setup(plan), plan)


def tffr_normal_apply(plan, image_in: torch.Tensor, image_out: torch.Tensor):
    _check(_abi.load().tffr_normal_apply(plan, _dev(image_in, "image_in", torch.complex64),
                                         _dev(image_out, "image_out", torch.complex64)), plan)


def tffr_weights_noalloc(lam_x: torch.Tensor, lam_y: torch.Tensor, Mx: int, My: int, D_out: torch.Tensor, *,
                         mode: str = "tffr", separable: bool = False, a: float = 0.01, q: float = 3.0,
                         tau: float = 0.97, user_D: torch.Tensor | None = None, count: bool = True, stream=None):
    """Weights without a plan and without device allocation, for callers that cannot
    allocate when they need them (see include/tffr.h).

    N is D_out's length.  lam_x (tFFR mode), lam_y (separable mode) and user_D (user
    mode) must hold at least N elements, and every tensor must sit on the current CUDA
    device: the kernel indexes them up to N on that device.  count=True reads the kept
    count back (a pageable copy and a stream synchronisation); under stream capture
    pass count=False.
    """
    if D_out.dim() != 1:
        raise ValueError("D_out must be 1-D")
    N = int(D_out.shape[0])
    needed = []
    if mode == "tffr":
        needed.append(("lam_x", lam_x))
        if separable:
            needed.append(("lam_y", lam_y))
    if mode == "user":
        if user_D is None:
            raise ValueError("user mode needs user_D")
        needed.append(("user_D", user_D))
    for name, t in needed:
        if t is None or t.dim() != 1 or int(t.shape[0]) < N:
            raise ValueError("%s must be 1-D with at least %d elements" % (name, N))
    if N:
        here = torch.cuda.current_device()
        for name, t in [("D_out", D_out), ("lam_x", lam_x), ("lam_y", lam_y), ("user_D", user_D)]:
            if t is not None and (not t.is_cuda or t.device.index != here):
                raise ValueError("%s must be on the current CUDA device (cuda:%d)" % (name, here))
    lib = _abi.load()
    o = _abi.tffr_weight_opts()
    lib.tffr_default_weight_opts(ctypes.byref(o))
    o.mode = WEIGHT_MODES[mode]
    o.separable = 1 if separable else 0
    o.a, o.q, o.tau = float(a), float(q), float(tau)
    if user_D is not None:
        o.user_D = _dev(user_D, "user_D", torch.float32).value
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
        self._check_values(values)
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        tffr_adjoint(self._handle(), values, out)
        return out

    def reconstruct(self, lam_x: torch.Tensor, lam_y: torch.Tensor, values: torch.Tensor,
                    out: torch.Tensor | None = None, **weight_opts) -> torch.Tensor:
        """set_points, weights and adjoint in one library call; keep references to the coordinates."""
        N = int(lam_x.shape[0])
        if values.dtype not in _VALUE_DTYPES[self.values]:
            raise TypeError("values dtype %s does not match the plan's %s" % (values.dtype, self.values))
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        self.N = None
        tffr_reconstruct(self._handle(), lam_x, lam_y, values, out, **weight_opts)
        self._coords = (lam_x, lam_y)
        self.N = N
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

    def _check_values(self, values: torch.Tensor):
        if values.dtype not in _VALUE_DTYPES[self.values]:
            raise TypeError("values dtype %s does not match the plan's %s" % (values.dtype, self.values))
        if self.N is not None and values.shape[0] != self.N:
            raise ValueError("expected %d samples, got %d" % (self.N, values.shape[0]))

    def adjoint_unweighted(self, values: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """E^H y, the Hermitian transpose of forward(apply_weights=False)."""
        self._check_values(values)
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        tffr_adjoint_unweighted(self._handle(), values, out)
        return out

    def weight_grad(self, grad_image: torch.Tensor, values: torch.Tensor,
                    out: torch.Tensor | None = None) -> torch.Tensor:
        """Re(conj(E grad_image) * values): the gradient of a real loss with respect to real weights."""
        self._check_values(values)
        if tuple(grad_image.shape) != (self.My, self.Mx):
            raise ValueError("grad_image must be [My, Mx] = [%d, %d]" % (self.My, self.Mx))
        if out is None:
            out = torch.empty(values.shape[0], dtype=torch.float32, device=self.device)
        tffr_weight_grad(self._handle(), grad_image, values, out)
        return out

    def cg(self, values: torch.Tensor, iters: int = 20, toeplitz: bool = False, out: torch.Tensor | None = None,
           residuals: bool = True):
        """Conjugate gradients on E^H D E f = E^H D y from f = 0 (every step in the library's kernels).
        Returns (f, residual norms for k = 0..iters, or None)."""
        self._check_values(values)
        if out is None:
            out = torch.empty((self.My, self.Mx), dtype=torch.complex64, device=self.device)
        hist = tffr_cg(self._handle(), values, out, iters, toeplitz, residuals)
        return out, hist

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
