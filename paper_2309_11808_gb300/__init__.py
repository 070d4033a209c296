"""GB300-native SPOD hot path (arXiv 2309.11808, Sec. 2.2) behind a C ABI.

``paper_2309_11808_gb300._lib`` mirrors include/spod.h entry for entry.  This
module adds ``SPOD``, a small convenience class that allocates outputs with
torch (device memory and streams only) and calls those entry points.  There is
no CPU path: without the built libspod.so and a CUDA device every call raises.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from ._lib import (SPOD_F32, SPOD_F64, SPOD_BF16, SPOD_C64, SPOD_C128,  # noqa: F401
                   SPOD_PREC_BF16, SPOD_PREC_BF16X3, SPOD_PREC_FP32, SPOD_PREC_FP64, SPOD_NORM_NB, SPOD_NORM_NB_MINUS_1, SPOD_WIN_HAMMING,
                   SPOD_WIN_HAMMING_PERIODIC, SPOD_WIN_HANN, SPOD_WIN_RECT, SPOD_WIN_USER, SpodError)

__all__ = ["SPOD", "SpodError", "make_desc"]

_DTYPES = {torch.float64: SPOD_F64, torch.float32: SPOD_F32, torch.bfloat16: SPOD_BF16,
           torch.complex64: SPOD_C64, torch.complex128: SPOD_C128}
_PRECS = {"fp64": SPOD_PREC_FP64, "fp32": SPOD_PREC_FP32, "bf16": SPOD_PREC_BF16, "bf16x3": SPOD_PREC_BF16X3}
_WINS = {"hamming": SPOD_WIN_HAMMING, "hamming_periodic": SPOD_WIN_HAMMING_PERIODIC, "hann": SPOD_WIN_HANN,
         "rect": SPOD_WIN_RECT, "user": SPOD_WIN_USER}
_NORMS = {"nb": SPOD_NORM_NB, "nb-1": SPOD_NORM_NB_MINUS_1}


def make_desc(npoints: int, nvars: int, nt: int, nfft: int, noverlap: int, *, dtype=torch.float32,
              precision: str = "fp32", window: str = "hamming", user_window=None, weights=None,
              norm: str = "nb", subtract_mean: bool = True, dt: float = 1.0, chunk_points: int = 0,
              mean_in_fft: bool = True):
    """Build an spod_plan_desc; returns (desc, keepalive) -- keep the second
    object alive until spod_plan_create has returned (it owns the host arrays)."""
    d = _lib.spod_desc_init()
    d.ndim = 1
    d.dims[0] = int(npoints)
    d.nvars = int(nvars)
    d.nt = int(nt)
    d.nfft = int(nfft)
    d.noverlap = int(noverlap)
    d.window = _WINS[window]
    d.in_dtype = _DTYPES[dtype]
    d.precision = _PRECS[precision]
    d.norm = _NORMS[norm]
    d.subtract_mean = int(bool(subtract_mean))
    d.dt = float(dt)
    d.chunk_points = int(chunk_points)
    d.mean_in_fft = int(bool(mean_in_fft))
    keep = []
    if user_window is not None:
        uw = np.ascontiguousarray(np.asarray(user_window, dtype=np.float64))
        keep.append(uw)
        d.user_window = uw.ctypes.data_as(_lib.C.POINTER(_lib.C.c_double))
    if weights is not None:
        w = weights.detach().cpu().numpy() if isinstance(weights, torch.Tensor) else weights
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        keep.append(w)
        d.weights = w.ctypes.data_as(_lib.C.POINTER(_lib.C.c_double))
    return d, keep


class SPOD:
    """One plan: ``fit(X)`` runs the hot path on a device tensor X[nt][M]."""

    def __init__(self, npoints: int, nvars: int, nt: int, nfft: int, noverlap: int | None = None, **kw):
        if noverlap is None:
            noverlap = nfft // 2
        desc, keep = make_desc(npoints, nvars, nt, nfft, noverlap, **kw)
        self.handle = _lib.spod_plan_create(desc)
        del keep
        info = _lib.spod_plan_get_info(self.handle)
        self.M, self.nb, self.nf, self.nt = info.M, info.nb, info.nf, info.nt
        self.info = info
        self.mean_in_fft = bool(info.mean_in_fft)
        self.f64 = desc.precision == SPOD_PREC_FP64

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.spod_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_x(self, X: torch.Tensor) -> None:
        if not X.is_cuda or not X.is_contiguous() or X.shape != (self.nt, self.M):
            raise ValueError(f"X must be a contiguous CUDA tensor of shape ({self.nt}, {self.M})")

    def fit(self, X: torch.Tensor, stream=None) -> "SPOD":
        self._check_x(X)
        _lib.spod_fit(self.handle, X, stream or torch.cuda.current_stream(X.device))
        return self

    def eigs(self, vectors: bool = False):
        lam = np.empty((self.nf, self.nb), dtype=np.float64)
        psi = np.empty((self.nf, self.nb, self.nb), dtype=np.complex128) if vectors else None
        _lib.spod_get_eigs(self.handle, lam, psi, on_device=False)
        return (lam, psi) if vectors else lam

    def gram(self) -> np.ndarray:
        g = np.empty((self.nf, self.nb, self.nb), dtype=np.complex128)
        _lib.spod_get_gram(self.handle, g)
        return g

    def freqs(self) -> np.ndarray:
        f = np.empty(self.nf, dtype=np.float64)
        _lib.spod_get_freqs(self.handle, f)
        return f

    def modes(self, X: torch.Tensor, nmodes: int | None = None, out: torch.Tensor | None = None, stream=None):
        self._check_x(X)
        nmodes = self.nb if nmodes is None else nmodes
        cdt = torch.complex128 if self.f64 else torch.complex64
        if out is None:
            out = torch.empty((self.nf, nmodes, self.M), dtype=cdt, device=X.device)
        _lib.spod_modes(self.handle, X, nmodes, out, stream or torch.cuda.current_stream(X.device))
        return out

    def sync(self, stream=None) -> None:
        _lib.spod_sync(self.handle, stream or torch.cuda.current_stream())


class SpodEigs(torch.autograd.Function):
    """lambda = SPOD eigenvalues of X ([nf][nb], FP64) with a hand-written adjoint.

    Forward: spod_fit.  Backward: spod_backward (the adjoint kernels carry
    dL/dlambda back through the Gram, the inverse DFT, the window, the
    overlap-add and the mean subtraction; Qhat is reused or recomputed, never
    stored per step).  Valid for simple eigenvalues.  The plan keeps the state
    of its last fit: run backward before fitting other data with the same plan.
    """

    @staticmethod
    def forward(ctx, X: torch.Tensor, plan: "SPOD"):
        plan.fit(X)
        lam = torch.empty((plan.nf, plan.nb), dtype=torch.float64, device=X.device)
        _lib.spod_get_eigs(plan.handle, lam, None, on_device=True)
        ctx.plan = plan
        ctx.save_for_backward(X)
        return lam

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (X,) = ctx.saved_tensors
        plan = ctx.plan
        dX = torch.empty(X.shape, dtype=torch.float64 if plan.f64 else torch.float32, device=X.device)
        _lib.spod_backward(plan.handle, g.detach().contiguous().to(torch.float64), X, dX,
                           torch.cuda.current_stream(X.device))
        return dX.to(X.dtype), None


def spod_eigs(X: torch.Tensor, plan: "SPOD") -> torch.Tensor:
    """Differentiable SPOD eigenvalues (see SpodEigs)."""
    return SpodEigs.apply(X, plan)


__all__ += ["SpodEigs", "spod_eigs"]
