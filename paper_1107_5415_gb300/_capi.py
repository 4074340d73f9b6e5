"""ctypes binding of the C ABI declared in include/pfft.h.

Each function here has the name of its C entry point and only marshals
arguments: Python ints / sequences become int64 arrays, device buffers are
passed as integer addresses, and a non-zero status raises ``PfftError``.
The library is built in-tree (``build_lib.py``); if it is missing or cannot
be loaded every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_lib

_lock = threading.Lock()
_lib = None

PFFT_C64, PFFT_C128 = 0, 1
PFFT_FLAG_TC_SPLIT = 1
PFFT_FLAG_LAYOUT_SNF = 2
PFFT_FLAG_AUTOTUNE = 4
PFFT_FLAG_TRANSPOSED = 8
PFFT_MAP_INPUT_BOX, PFFT_MAP_OUTPUT_BOX, PFFT_MAP_INPUT_SNF, PFFT_MAP_OUTPUT_SNF = 0, 1, 2, 3
PWT_DIRICHLET, PWT_DLVP = 0, 1
PWT_FLAG_INPUT_SNF = 1
PFFT_BATCH_NO_GRAPH, PFFT_BATCH_AUTOTUNE, PFFT_BATCH_RADIX8, PFFT_BATCH_ONE_LAUNCH = 1, 2, 4, 8

STATUS = {0: "PFFT_OK", 1: "PFFT_ERR_ARG", 2: "PFFT_ERR_SINGULAR", 3: "PFFT_ERR_OVERFLOW",
          4: "PFFT_ERR_NOT_INTEGRAL", 5: "PFFT_ERR_UNSUPPORTED", 6: "PFFT_ERR_OOM", 7: "PFFT_ERR_CUDA",
          8: "PFFT_ERR_TIMEOUT", 9: "PFFT_ERR_DEVICE_CHECK"}


class PfftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS.get(status, str(status))
        try:
            msg = lib().pfft_status_string(status).decode()
        except Exception:  # pragma: no cover - only if the library itself is broken
            msg = ""
        super().__init__(f"{where}: {name} ({msg})")


_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

_SIGS = {
    "pfft_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pfft_hermite_normal_form": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p]),
    "pfft_smith_normal_form": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p, _i64p, _i64p]),
    "pfft_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_uint]),
    "pfft_plan_info": (ctypes.c_int, [_vp, _i64p, ctypes.POINTER(ctypes.c_int), _i64p, _i64p, _i64p]),
    "pfft_plan_route": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pfft_index_map": (ctypes.c_int, [_vp, ctypes.c_int, _i64p]),
    "pfft_device_index_map": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "pfft_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pfft_inverse": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pfft_plan_destroy": (ctypes.c_int, [_vp]),
    "pfft_last_device_status": (ctypes.c_int, [_vp, _vp]),
    "pfft_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pfft_batch_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pfft_batch_device_status": (ctypes.c_int, [_vp, _vp]),
    "pfft_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pfft_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_char_p), _i64p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "pwt_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.c_int, _i64p,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_uint]),
    "pwt_plan_info": (ctypes.c_int, [_vp, ctypes.c_int, _i64p, _i64p]),
    "pwt_decompose": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(_vp), _vp]),
    "pwt_reconstruct": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp), _vp, _vp]),
    "pwt_adjoint": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp), _vp, _vp]),
    "pwt_plan_destroy": (ctypes.c_int, [_vp]),
    "pwt_decompose_noalloc": (ctypes.c_int, [ctypes.c_int, _i64p, ctypes.c_int, _i64p, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int64, _vp, _vp, ctypes.POINTER(_vp),
                                             _vp]),
    "pfft_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p,
                                         _i64p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint]),
    "pfft_batch_info": (ctypes.c_int, [_vp, _i64p, _i64p]),
    "pfft_batch_split_layout": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _i64p, _i64p, _i64p, _i64p]),
    "pfft_batch_schedule": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pfft_batch_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pfft_batch_destroy": (ctypes.c_int, [_vp]),
    "pwt_split_general": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p, ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp,
                                         _vp]),
    "pwt_merge_general": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p, ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp,
                                         _vp]),
}


def declared_symbols():
    """Names of the entry points this binding expects the library to export."""
    return sorted(_SIGS)


def lib(build: bool = True):
    """Load (building first if needed) the in-tree library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib.build() if build else build_lib.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"pattern FFT library not built: {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise PfftError(st, where)


def _i64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return a, a.ctypes.data_as(_i64p)


def _mat(M):
    A = np.asarray(M, dtype=np.int64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("M must be a square integer matrix")
    return A.shape[0], _i64(A.reshape(-1))


# ------------------------------------------------------------ host queries
def pfft_hermite_normal_form(M):
    d, (a, p) = _mat(M)
    H, hp = _i64(np.zeros(d * d))
    _check(lib().pfft_hermite_normal_form(d, p, hp), "pfft_hermite_normal_form")
    return H.reshape(d, d)


def pfft_smith_normal_form(M):
    d, (a, p) = _mat(M)
    Q, qp = _i64(np.zeros(d * d))
    E, ep = _i64(np.zeros(d))
    R, rp = _i64(np.zeros(d * d))
    _check(lib().pfft_smith_normal_form(d, p, qp, ep, rp), "pfft_smith_normal_form")
    return Q.reshape(d, d), E, R.reshape(d, d)


# ------------------------------------------------------------ FFT plans
def pfft_plan_create(M, batch: int, dtype: int = PFFT_C64, flags: int = 0):
    d, (a, p) = _mat(M)
    h = _vp()
    _check(lib().pfft_plan_create(ctypes.byref(h), d, p, int(batch), int(dtype), int(flags)),
           "pfft_plan_create")
    return h.value


def pfft_plan_info(plan, d: int):
    m = ctypes.c_int64()
    dM = ctypes.c_int()
    eps, ep = _i64(np.zeros(d))
    ib, ip = _i64(np.zeros(d))
    ob, op = _i64(np.zeros(d))
    _check(lib().pfft_plan_info(plan, ctypes.byref(m), ctypes.byref(dM), ep, ip, op), "pfft_plan_info")
    return m.value, dM.value, eps, ib, ob


def pfft_plan_route(plan):
    fwd, inv = ctypes.c_int(), ctypes.c_int()
    _check(lib().pfft_plan_route(plan, ctypes.byref(fwd), ctypes.byref(inv)), "pfft_plan_route")
    return bool(fwd.value), bool(inv.value)


def pfft_index_map(plan, which: int, m: int, width: int):
    out, op = _i64(np.zeros(m * width))
    _check(lib().pfft_index_map(plan, int(which), op), "pfft_index_map")
    return out.reshape(m, width)


def pfft_device_index_map(plan, which: int, slots_ptr: int, stream: int):
    _check(lib().pfft_device_index_map(plan, int(which), slots_ptr, stream), "pfft_device_index_map")


def pfft_forward(plan, in_ptr: int, out_ptr: int, stream: int):
    _check(lib().pfft_forward(plan, in_ptr, out_ptr, stream), "pfft_forward")


def pfft_inverse(plan, in_ptr: int, out_ptr: int, stream: int):
    _check(lib().pfft_inverse(plan, in_ptr, out_ptr, stream), "pfft_inverse")


def pfft_last_device_status(plan, stream: int):
    """Status word of the plan's kernels (0 = ok); raises on a non-zero status."""
    _check(lib().pfft_last_device_status(plan, stream), "pfft_last_device_status")


def pfft_set_wait_limit(plan, spins: int):
    """Iteration limit of the row pass's first bounded wait (< 0: default)."""
    _check(lib().pfft_set_wait_limit(plan, int(spins)), "pfft_set_wait_limit")


def pfft_plan_destroy(plan):
    _check(lib().pfft_plan_destroy(plan), "pfft_plan_destroy")


def pfft_profile_enable(plan, enable: bool):
    _check(lib().pfft_profile_enable(plan, 1 if enable else 0), "pfft_profile_enable")


def pfft_profile_read(plan, cap: int = 8):
    names = (ctypes.c_char_p * cap)()
    launches, lp = _i64(np.zeros(cap))
    ms = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    _check(lib().pfft_profile_read(plan, names, lp, ms, cap, ctypes.byref(n)), "pfft_profile_read")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n.value)}


# ------------------------------------------------------------ wavelet plans
def pwt_plan_create(M, Js, symbol: int, eta: float, batch: int, dtype: int = PFFT_C64, flags: int = 0):
    d, (a, p) = _mat(M)
    Ja = np.asarray(Js, dtype=np.int64)
    levels = Ja.shape[0]
    if Ja.shape != (levels, d, d):
        raise ValueError("J must have shape [levels, d, d]")
    ja, jp = _i64(Ja.reshape(-1))
    h = _vp()
    _check(lib().pwt_plan_create(ctypes.byref(h), d, p, levels, jp, int(symbol), float(eta), int(batch),
                                 int(dtype), int(flags)), "pwt_plan_create")
    return h.value


def pwt_plan_info(plan, level: int, d: int):
    n = ctypes.c_int64()
    box, bp = _i64(np.zeros(d))
    _check(lib().pwt_plan_info(plan, int(level), ctypes.byref(n), bp), "pwt_plan_info")
    return n.value, box


def _ptr_array(ptrs):
    arr = (_vp * len(ptrs))(*[_vp(int(x)) for x in ptrs])
    return arr


def pwt_decompose(plan, c_hat_ptr: int, scaling_ptr: int, wavelet_ptrs, stream: int):
    arr = _ptr_array(wavelet_ptrs)
    _check(lib().pwt_decompose(plan, c_hat_ptr, scaling_ptr, arr, stream), "pwt_decompose")


def pwt_reconstruct(plan, scaling_ptr: int, wavelet_ptrs, c_hat_ptr: int, stream: int):
    arr = _ptr_array(wavelet_ptrs)
    _check(lib().pwt_reconstruct(plan, scaling_ptr, arr, c_hat_ptr, stream), "pwt_reconstruct")


def pwt_adjoint(plan, scaling_ptr: int, wavelet_ptrs, c_hat_ptr: int, stream: int):
    arr = _ptr_array(wavelet_ptrs)
    _check(lib().pwt_adjoint(plan, scaling_ptr, arr, c_hat_ptr, stream), "pwt_adjoint")


def pwt_plan_destroy(plan):
    _check(lib().pwt_plan_destroy(plan), "pwt_plan_destroy")


def pwt_decompose_noalloc(M, Js, symbol: int, eta: float, batch: int, c_hat_ptr: int, scaling_ptr: int,
                          wavelet_ptrs, stream: int):
    """Plan-free decomposition that allocates no device memory (complex64)."""
    d, (a, p) = _mat(M)
    Ja = np.asarray(Js, dtype=np.int64)
    levels = Ja.shape[0]
    if Ja.shape != (levels, d, d):
        raise ValueError("J must have shape [levels, d, d]")
    if len(wavelet_ptrs) != levels:
        raise ValueError("need one wavelet pointer per level")
    ja, jp = _i64(Ja.reshape(-1))
    arr = _ptr_array(wavelet_ptrs)
    _check(lib().pwt_decompose_noalloc(d, p, levels, jp, int(symbol), float(eta), int(batch), c_hat_ptr,
                                       scaling_ptr, arr, stream), "pwt_decompose_noalloc")


# ------------------------------------------------------------ pattern batches
def pfft_batch_create(Ms, Js=None, symbol: int = PWT_DIRICHLET, eta: float = 0.125, dtype: int = PFFT_C64,
                      flags: int = 0):
    """Ms: sequence of square integer matrices (any mix of d); Js: None or one
    dilation per pattern, each of its pattern's d."""
    ds = [int(np.asarray(M).shape[0]) for M in Ms]
    for M, d in zip(Ms, ds):
        if np.asarray(M).shape != (d, d):
            raise ValueError("every M must be square")
    d_arr = (ctypes.c_int * len(ds))(*ds)
    ma, mp = _i64(np.concatenate([np.asarray(M, dtype=np.int64).reshape(-1) for M in Ms]))
    jp = None
    if Js is not None:
        if len(Js) != len(Ms):
            raise ValueError("one dilation per pattern is required")
        for J, d in zip(Js, ds):
            if np.asarray(J).shape != (d, d):
                raise ValueError("each J must have the shape of its M")
        ja, jp = _i64(np.concatenate([np.asarray(J, dtype=np.int64).reshape(-1) for J in Js]))
    h = _vp()
    _check(lib().pfft_batch_create(ctypes.byref(h), len(ds), d_arr, mp, jp, int(symbol), float(eta), int(dtype),
                                   int(flags)), "pfft_batch_create")
    return h.value


def pfft_batch_info(batch, n: int):
    m, mp = _i64(np.zeros(n))
    total = ctypes.c_int64()
    _check(lib().pfft_batch_info(batch, mp, ctypes.byref(total)), "pfft_batch_info")
    return m, total.value


def pfft_batch_split_layout(batch, n: int):
    """(p [n], scaling offsets [n], wavelet offsets [n], scaling total, wavelet total)."""
    p = (ctypes.c_int * n)()
    so = np.zeros(n, dtype=np.int64)
    wo = np.zeros(n, dtype=np.int64)
    st, wt = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().pfft_batch_split_layout(batch, p, so.ctypes.data_as(_i64p), wo.ctypes.data_as(_i64p),
                                         ctypes.byref(st), ctypes.byref(wt)), "pfft_batch_split_layout")
    return np.array(list(p), dtype=np.int64), so, wo, int(st.value), int(wt.value)


def pfft_batch_schedule(batch):
    r, c, o, x = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().pfft_batch_schedule(batch, ctypes.byref(r), ctypes.byref(c), ctypes.byref(o), ctypes.byref(x)),
           "pfft_batch_schedule")
    return r.value, c.value, o.value, x.value


def pfft_batch_forward(batch, in_ptr: int, c_hat_ptr: int, scaling_ptr, wavelet_ptr, stream: int):
    _check(lib().pfft_batch_forward(batch, in_ptr, c_hat_ptr, scaling_ptr, wavelet_ptr, stream),
           "pfft_batch_forward")


def pfft_batch_set_wait_limit(batch, spins: int):
    """Tries of every dependency wait of a single-launch batch (< 0: default)."""
    _check(lib().pfft_batch_set_wait_limit(batch, int(spins)), "pfft_batch_set_wait_limit")


def pfft_batch_device_status(batch, stream: int):
    """Reads and clears the batch's device status word; raises on PFFT_ERR_TIMEOUT."""
    _check(lib().pfft_batch_device_status(batch, stream), "pfft_batch_device_status")


def pfft_batch_destroy(batch):
    _check(lib().pfft_batch_destroy(batch), "pfft_batch_destroy")


# ------------------------------------------------------------ general split step
def _mj(M, J):
    d, (a, p) = _mat(M)
    dj, (b, q) = _mat(J)
    if dj != d:
        raise ValueError("M and J must have the same size")
    return d, a, p, b, q


def pwt_split_general(M, J, batch: int, dtype: int, symbols_ptr: int, c_hat_ptr: int, parts_ptr: int, stream: int):
    d, a, p, b, q = _mj(M, J)
    _check(lib().pwt_split_general(d, p, q, int(batch), int(dtype), symbols_ptr, c_hat_ptr, parts_ptr, stream),
           "pwt_split_general")


def pwt_merge_general(M, J, batch: int, dtype: int, symbols_ptr: int, parts_ptr: int, c_hat_ptr: int, stream: int):
    d, a, p, b, q = _mj(M, J)
    _check(lib().pwt_merge_general(d, p, q, int(batch), int(dtype), symbols_ptr, parts_ptr, c_hat_ptr, stream),
           "pwt_merge_general")
