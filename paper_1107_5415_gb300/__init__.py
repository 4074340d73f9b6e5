"""GB300 pattern FFT and fast wavelet split (sm_103a).

The Fourier transform on the pattern P(M) of a regular integer matrix M
(eq. (Fouriermatrix), Section 2.2) and the wavelet split step built on it
(Section 5.3, step 4; Dirichlet symbols of Section 6.2), computed by
hand-written CUDA kernels behind the C ABI of ``include/pfft.h``.

PyTorch supplies device memory, streams and autograd only; every step of the
transform runs in the library's kernels.  If the library cannot be loaded,
every operation raises -- there is no CPU fallback.

Layout: a signal on P(M) is a complex tensor ``[batch, m]`` whose slot s holds
the value at y = box point s of the Hermite normal form H(M) (row-major, last
coordinate fastest); Fourier coefficients are stored the same way over the box
of H(M^T).  ``PatternFFT.index_map`` returns those coordinates.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _capi
from ._capi import (PFFT_BATCH_AUTOTUNE, PFFT_BATCH_NO_GRAPH, PFFT_BATCH_ONE_LAUNCH, PFFT_BATCH_RADIX8, PFFT_C64, PFFT_C128, PFFT_FLAG_LAYOUT_SNF,
                    pfft_batch_device_status, pfft_batch_set_wait_limit, pfft_batch_split_layout,
                    PFFT_FLAG_AUTOTUNE, PFFT_FLAG_TC_SPLIT, PFFT_FLAG_TRANSPOSED,
                    PFFT_MAP_INPUT_BOX,
                    PFFT_MAP_INPUT_SNF, PFFT_MAP_OUTPUT_BOX, PFFT_MAP_OUTPUT_SNF, PWT_DIRICHLET, PWT_DLVP,
                    PWT_FLAG_INPUT_SNF,
                    PfftError, pfft_batch_create, pfft_batch_destroy, pfft_batch_forward, pfft_batch_info,
                    pfft_batch_schedule, pfft_device_index_map, pwt_merge_general, pwt_split_general,
                    pfft_forward, pfft_hermite_normal_form, pfft_index_map, pfft_inverse, pfft_plan_create,
                    pfft_last_device_status, pfft_plan_destroy, pfft_plan_info, pfft_plan_route, pfft_profile_enable, pfft_profile_read,
                    pfft_set_wait_limit, pfft_smith_normal_form, pwt_adjoint, pwt_decompose, pwt_plan_create, pwt_plan_destroy,
                    pwt_plan_info, pwt_reconstruct)

__all__ = [
    "PatternFFT", "WaveletSplit", "PatternBatch", "pattern_fft", "pattern_ifft", "wavelet_decompose",
    "PFFT_BATCH_NO_GRAPH", "PFFT_BATCH_AUTOTUNE", "PFFT_BATCH_RADIX8", "PFFT_BATCH_ONE_LAUNCH",
    "pfft_batch_set_wait_limit", "pfft_batch_device_status", "PFFT_FLAG_TC_SPLIT", "PFFT_FLAG_LAYOUT_SNF", "PWT_FLAG_INPUT_SNF", "pfft_batch_create", "pfft_batch_info",
    "pfft_batch_schedule", "pfft_batch_split_layout", "pfft_batch_forward", "pfft_batch_destroy", "split_general", "merge_general",
    "pwt_split_general", "pwt_merge_general",
    "PfftError", "PFFT_C64", "PFFT_C128", "PWT_DIRICHLET", "PWT_DLVP",
    "PFFT_MAP_INPUT_BOX", "PFFT_MAP_OUTPUT_BOX", "PFFT_MAP_INPUT_SNF", "PFFT_MAP_OUTPUT_SNF",
    "PFFT_FLAG_AUTOTUNE", "PFFT_FLAG_TRANSPOSED", "pfft_plan_route",
    "pfft_plan_create", "pfft_plan_info", "pfft_index_map", "pfft_device_index_map", "pfft_forward",
    "pfft_inverse", "pfft_plan_destroy", "pfft_last_device_status", "pfft_set_wait_limit", "pfft_profile_enable", "pfft_profile_read",
    "pfft_hermite_normal_form", "pfft_smith_normal_form", "pwt_plan_create", "pwt_plan_info",
    "pwt_decompose", "pwt_reconstruct", "pwt_adjoint", "pwt_plan_destroy", "library_path",
]


def library_path() -> str:
    """Path of the loaded shared library (building it first if needed)."""
    _capi.lib()
    return _capi.build_lib.LIB


def _dtype_code(dtype) -> int:
    if dtype == torch.complex64:
        return PFFT_C64
    if dtype == torch.complex128:
        return PFFT_C128
    raise ValueError("dtype must be torch.complex64 or torch.complex128")


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_tensor(x: torch.Tensor, dtype, shape, name: str):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if tuple(x.shape) != tuple(shape) or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous tensor of shape {tuple(shape)}")


class PatternFFT:
    """Plan of the transform on P(M) for ``batch`` signals (wraps pfft_plan)."""

    def __init__(self, M, batch: int = 1, dtype=torch.complex64, tc_split: bool = False, layout: str = "box",
                 route: str = "direct"):
        """``tc_split``: run the radix-16 / 32 stages on the tensor cores in
        split fp16 (PFFT_FLAG_TC_SPLIT; complex64 only).  ``layout``: "box"
        (Hermite boxes, the default) or "snf" (Smith coordinates,
        PFFT_FLAG_LAYOUT_SNF).  ``route``: "direct" (the passes of M),
        "auto" (each direction through the plan of M^T where that measures
        faster, PFFT_FLAG_AUTOTUNE) or "transposed" (both directions through
        it, PFFT_FLAG_TRANSPOSED)."""
        if layout not in ("box", "snf"):
            raise ValueError('layout must be "box" or "snf"')
        if route not in ("direct", "auto", "transposed"):
            raise ValueError('route must be "direct", "auto" or "transposed"')
        self.M = np.asarray(M, dtype=np.int64)
        self.d = int(self.M.shape[0])
        self.batch = int(batch)
        self.dtype = dtype
        self.tc_split = bool(tc_split)
        self.layout = layout
        flags = (PFFT_FLAG_TC_SPLIT if tc_split else 0) | (PFFT_FLAG_LAYOUT_SNF if layout == "snf" else 0)
        flags |= {"direct": 0, "auto": PFFT_FLAG_AUTOTUNE, "transposed": PFFT_FLAG_TRANSPOSED}[route]
        self._h = pfft_plan_create(self.M, self.batch, _dtype_code(dtype), flags)
        self.m, self.dM, self.eps, self.in_box, self.out_box = pfft_plan_info(self._h, self.d)

    @property
    def shape(self):
        return (self.batch, self.m)

    @property
    def route(self):
        """(forward, inverse): True where the direction runs through the plan of M^T."""
        return pfft_plan_route(self._h)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """c_hat = F(M) c: x on the box of H(M), result on the box of H(M^T)."""
        _check_tensor(x, self.dtype, self.shape, "input")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=x.device)
        _check_tensor(out, self.dtype, self.shape, "output")
        pfft_forward(self._h, x.data_ptr(), out.data_ptr(), _stream(stream))
        return out

    def inverse(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """c = F(M)^H c_hat (F(M) is unitary)."""
        _check_tensor(x, self.dtype, self.shape, "input")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=x.device)
        _check_tensor(out, self.dtype, self.shape, "output")
        pfft_inverse(self._h, x.data_ptr(), out.data_ptr(), _stream(stream))
        return out

    def index_map(self, which: int) -> np.ndarray:
        width = self.d if which in (PFFT_MAP_INPUT_BOX, PFFT_MAP_OUTPUT_BOX) else max(self.dM, 1)
        return pfft_index_map(self._h, which, self.m, width)

    def device_index_map(self, which: int, device=None) -> torch.Tensor:
        out = torch.empty(self.m, dtype=torch.int64, device=device or "cuda")
        pfft_device_index_map(self._h, which, out.data_ptr(), _stream(None))
        return out

    def check_device_status(self, stream=None):
        """Raise PfftError if a kernel of this plan recorded a device-side failure."""
        pfft_last_device_status(self._h, _stream(stream))

    def profile(self, enable: bool = True):
        pfft_profile_enable(self._h, enable)

    def profile_read(self):
        return pfft_profile_read(self._h)

    def close(self):
        if getattr(self, "_h", None):
            pfft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _FFTFn(torch.autograd.Function):
    """y = F c with the hand-written adjoint: dL/dc = F^H dL/dy (= inverse)."""

    @staticmethod
    def forward(ctx, x, plan, inverse):
        ctx.plan = plan
        ctx.inverse = inverse
        x = x.contiguous()
        return plan.inverse(x) if inverse else plan.forward(x)

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        # F is unitary, so its adjoint is its inverse (and vice versa).
        return (ctx.plan.forward(g) if ctx.inverse else ctx.plan.inverse(g)), None, None


def pattern_fft(x: torch.Tensor, plan: PatternFFT) -> torch.Tensor:
    """Differentiable forward transform."""
    return _FFTFn.apply(x, plan, False)


def pattern_ifft(x: torch.Tensor, plan: PatternFFT) -> torch.Tensor:
    """Differentiable inverse transform."""
    return _FFTFn.apply(x, plan, True)


class WaveletSplit:
    """Plan of ``levels`` split steps (wraps pwt_plan)."""

    def __init__(self, M, Js, symbol: int = PWT_DIRICHLET, eta: float = 0.125, batch: int = 1,
                 dtype=torch.complex64, input_layout: str = "box"):
        """``input_layout``: "box" (default) or "snf" -- the first level's
        coefficients in the Smith-coordinate order of a ``PatternFFT(M,
        layout="snf")`` output (PWT_FLAG_INPUT_SNF)."""
        if input_layout not in ("box", "snf"):
            raise ValueError('input_layout must be "box" or "snf"')
        self.M = np.asarray(M, dtype=np.int64)
        self.d = int(self.M.shape[0])
        self.Js = np.asarray(Js, dtype=np.int64)
        self.levels = int(self.Js.shape[0])
        self.batch = int(batch)
        self.dtype = dtype
        self.input_layout = input_layout
        self._h = pwt_plan_create(self.M, self.Js, symbol, eta, self.batch, _dtype_code(dtype),
                                  PWT_FLAG_INPUT_SNF if input_layout == "snf" else 0)
        self.sizes = []
        self.boxes = []
        for lev in range(self.levels + 1):
            n, box = pwt_plan_info(self._h, lev, self.d)
            self.sizes.append(n)
            self.boxes.append(box)

    def decompose(self, c_hat: torch.Tensor, stream=None):
        """Returns (scaling [batch, n_L], [wavelet_l [batch, n_l] for l = 1..L])."""
        _check_tensor(c_hat, self.dtype, (self.batch, self.sizes[0]), "c_hat")
        dev = c_hat.device
        wav = [torch.empty((self.batch, self.sizes[l + 1]), dtype=self.dtype, device=dev)
               for l in range(self.levels)]
        sc = torch.empty((self.batch, self.sizes[-1]), dtype=self.dtype, device=dev)
        pwt_decompose(self._h, c_hat.data_ptr(), sc.data_ptr(), [w.data_ptr() for w in wav], _stream(stream))
        return sc, wav

    def _synth(self, fn, scaling, wavelets, stream):
        _check_tensor(scaling, self.dtype, (self.batch, self.sizes[-1]), "scaling")
        if len(wavelets) != self.levels:
            raise ValueError("one wavelet part per level is required")
        for l, w in enumerate(wavelets):
            _check_tensor(w, self.dtype, (self.batch, self.sizes[l + 1]), f"wavelet[{l}]")
        out = torch.empty((self.batch, self.sizes[0]), dtype=self.dtype, device=scaling.device)
        fn(self._h, scaling.data_ptr(), [w.data_ptr() for w in wavelets], out.data_ptr(), _stream(stream))
        return out

    def reconstruct(self, scaling, wavelets, stream=None):
        return self._synth(pwt_reconstruct, scaling, wavelets, stream)

    def adjoint(self, scaling, wavelets, stream=None):
        return self._synth(pwt_adjoint, scaling, wavelets, stream)

    def close(self):
        if getattr(self, "_h", None):
            pwt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PatternBatch:
    """Many patterns of uneven size, transformed (and split one level) together
    (wraps pfft_batch).  Signals are concatenated: pattern i owns elements
    ``offsets[i] : offsets[i] + m[i]`` of the input and of ``c_hat``.  With
    dilations J_i of determinant p_i, the scaling part of pattern i is
    ``scaling[sc_off[i] : sc_off[i] + m[i] / p[i]]`` and its p_i - 1 band
    parts are consecutive in ``wavelet`` from ``wv_off[i]`` (for p_i = 2 both
    offsets are offsets[i] // 2)."""

    def __init__(self, Ms, Js=None, symbol: int = PWT_DIRICHLET, eta: float = 0.125, dtype=torch.complex64,
                 flags: int = 0):
        self.n = len(Ms)
        self.dtype = dtype
        self.has_split = Js is not None
        self._h = pfft_batch_create(Ms, Js, symbol, eta, _dtype_code(dtype), flags)
        self.m, self.total = pfft_batch_info(self._h, self.n)
        self.offsets = np.concatenate([[0], np.cumsum(self.m)[:-1]]).astype(np.int64)
        self.p, self.sc_off, self.wv_off, self.sc_total, self.wv_total = pfft_batch_split_layout(self._h, self.n)

    def schedule(self):
        """(row tile budget, column tile budget, order, largest power-of-two radix) chosen at creation."""
        return pfft_batch_schedule(self._h)

    def forward(self, x: torch.Tensor, c_hat=None, scaling=None, wavelet=None, split: bool = True, stream=None):
        """Returns c_hat, or (c_hat, scaling, wavelet) when the batch has dilations and ``split``."""
        _check_tensor(x, self.dtype, (self.total,), "input")
        dev = x.device
        if c_hat is None:
            c_hat = torch.empty(self.total, dtype=self.dtype, device=dev)
        _check_tensor(c_hat, self.dtype, (self.total,), "c_hat")
        if not (self.has_split and split):
            pfft_batch_forward(self._h, x.data_ptr(), c_hat.data_ptr(), None, None, _stream(stream))
            return c_hat
        if scaling is None:
            scaling = torch.empty(self.sc_total, dtype=self.dtype, device=dev)
        if wavelet is None:
            wavelet = torch.empty(self.wv_total, dtype=self.dtype, device=dev)
        _check_tensor(scaling, self.dtype, (self.sc_total,), "scaling")
        _check_tensor(wavelet, self.dtype, (self.wv_total,), "wavelet")
        pfft_batch_forward(self._h, x.data_ptr(), c_hat.data_ptr(), scaling.data_ptr(), wavelet.data_ptr(),
                           _stream(stream))
        return c_hat, scaling, wavelet

    def set_wait_limit(self, spins: int):
        """PFFT_BATCH_ONE_LAUNCH batches: tries of every dependency wait (< 0: default)."""
        pfft_batch_set_wait_limit(self._h, spins)

    def check_device_status(self, stream=None):
        """Raise PfftError if a wait of the single launch gave up (reads and clears the status)."""
        pfft_batch_device_status(self._h, _stream(stream))

    def close(self):
        if getattr(self, "_h", None):
            pfft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _det_int(A) -> int:
    A = np.asarray(A, dtype=np.int64)
    return int(round(abs(np.linalg.det(A.astype(np.float64)))))


def split_general(M, J, symbols, c_hat: torch.Tensor, stream=None) -> torch.Tensor:
    """Section 5.3 step 4 for |det J| = p (cyclic G(J^T)): c_hat
    [batch, |det M|] -> parts [p, batch, |det M| / p].  ``symbols``: the
    caller's symbols [p, |det M|] (p <= 16), or None for the built-in
    unitary band system (periodised Dirichlet scaling symbol and its
    completion; any p)."""
    batch, m = c_hat.shape
    p = symbols.shape[0] if symbols is not None else _det_int(J)
    _check_tensor(c_hat, c_hat.dtype, (batch, m), "c_hat")
    if symbols is not None:
        _check_tensor(symbols, c_hat.dtype, (p, m), "symbols")
    out = torch.empty((p, batch, m // p), dtype=c_hat.dtype, device=c_hat.device)
    pwt_split_general(M, J, batch, _dtype_code(c_hat.dtype), symbols.data_ptr() if symbols is not None else 0,
                      c_hat.data_ptr(), out.data_ptr(), _stream(stream))
    return out


def merge_general(M, J, symbols, parts: torch.Tensor, stream=None) -> torch.Tensor:
    """Adjoint of ``split_general`` (its inverse for unitary symbol systems,
    the built-in one included: ``symbols`` None)."""
    p, batch, n = parts.shape
    m = p * n
    _check_tensor(parts, parts.dtype, (p, batch, n), "parts")
    if symbols is not None:
        _check_tensor(symbols, parts.dtype, (p, m), "symbols")
    out = torch.empty((batch, m), dtype=parts.dtype, device=parts.device)
    pwt_merge_general(M, J, batch, _dtype_code(parts.dtype), symbols.data_ptr() if symbols is not None else 0,
                      parts.data_ptr(), out.data_ptr(), _stream(stream))
    return out


class _SplitFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c_hat, plan):
        ctx.plan = plan
        sc, wav = plan.decompose(c_hat.contiguous())
        return (sc, *wav)

    @staticmethod
    def backward(ctx, g_sc, *g_wav):
        plan = ctx.plan
        z = lambda t, n: torch.zeros((plan.batch, n), dtype=plan.dtype, device="cuda") if t is None \
            else t.contiguous()
        g_sc = z(g_sc, plan.sizes[-1])
        g_wav = [z(g, plan.sizes[l + 1]) for l, g in enumerate(g_wav)]
        return plan.adjoint(g_sc, g_wav), None


def wavelet_decompose(c_hat: torch.Tensor, plan: WaveletSplit):
    """Differentiable multi-level split; backward runs the adjoint kernels."""
    out = _SplitFn.apply(c_hat, plan)
    return out[0], list(out[1:])
