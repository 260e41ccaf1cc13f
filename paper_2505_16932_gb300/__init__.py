"""Polar Express on GB300: Python binding of the C-ABI library.

Argument marshalling only; every step of the online stage runs in the
library's CUDA kernels. The names follow the C ABI (include/polar_express.h):

* ``pe_coeffs(degree, l, T, safety)``: offline FP64 coefficient table
  (Thm. 1 greedy minimax composition, Alg. 3 Remez, App. A stabilisations).
* ``pe_polar(X, table, dtype)``: polar factor of one CUDA tensor, in place.
* ``pe_polar_batched(Xs, table, dtype)``: a list of CUDA tensors of uneven
  shapes, one persistent grouped launch per polynomial step in a cached
  CUDA graph.

PyTorch is used only for device memory and streams. If the shared library is
missing the binding raises; it never falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

PE_OK, PE_EINVAL, PE_ENOMEM, PE_ECUDA, PE_ENOCONV, PE_ETIMEOUT, PE_EUNSUPPORTED = range(7)
PE_FP32, PE_BF16, PE_BF16X3 = 0, 1, 2
PE_IO_FP32, PE_IO_BF16 = 0, 1
PE_SAFETY_SKIP_LAST = 1
PE_BATCH_NO_GRAPH, PE_BATCH_NO_TUNE, PE_BATCH_PHASED = 1, 2, 4

DTYPES = {"fp32": PE_FP32, "bf16": PE_BF16, "bf16x3": PE_BF16X3}
_STATUS = {0: "PE_OK", 1: "PE_EINVAL", 2: "PE_ENOMEM", 3: "PE_ECUDA", 4: "PE_ENOCONV",
           5: "PE_ETIMEOUT", 6: "PE_EUNSUPPORTED"}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "polar_express.h")


class PolarExpressError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def library_path() -> str:
    return _build.library_path()


def lib() -> ctypes.CDLL:
    """Load the shared library (it must have been built with build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise PolarExpressError(PE_EUNSUPPORTED,
                                f"{path} is missing; build it with paper_2505_16932_gb300.build.build()")
    L = ctypes.CDLL(path)
    c_d, c_i, c_u, c_p, c_i64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_void_p, ctypes.c_int64
    P_d = ctypes.POINTER(c_d)
    P_i = ctypes.POINTER(c_i)
    P_i64 = ctypes.POINTER(c_i64)
    sig = {
        "pe_version": (c_i, []),
        "pe_coeffs": (c_i, [c_i, c_d, c_i, c_d, P_d, P_d]),
        "pe_coeffs_ex": (c_i, [c_i, c_d, c_i, c_d, c_d, c_u, P_d, P_d, P_i]),
        "pe_polar": (c_i, [c_p, c_i64, c_i64, P_d, c_i, c_i, c_p]),
        "pe_polar_ex": (c_i, [c_p, c_i64, c_i64, c_i64, c_i, P_d, c_i, c_i, c_d, c_d, c_p]),
        "pe_polar_batched": (c_i, [ctypes.POINTER(c_p), P_i64, P_i64, c_i, P_d, c_i, c_i, c_p]),
        "pe_polar_batched_ex": (c_i, [ctypes.POINTER(c_p), P_i64, P_i64, c_i, c_i, P_d, c_i, c_i, c_d, c_d,
                                      c_u, c_p]),
        "pe_sync_status": (c_i, [c_p]),
        "pe_launch_count": (c_i64, []),
        "pe_last_error": (ctypes.c_char_p, []),
        "pe_release": (None, []),
        "pe_debug_set": (c_i, [c_i, c_i64]),
        "pe_trace_enable": (c_i, [c_i]),
        "pe_trace_read": (c_i, [P_i64, P_d, c_i]),
        "pe_polar_batched_host": (c_i, [ctypes.POINTER(c_p), ctypes.POINTER(c_p), P_i64, P_i64, c_i, P_d, c_i, c_i,
                                        c_i, c_p]),
        "pe_muon_batched": (c_i, [ctypes.POINTER(c_p), ctypes.POINTER(c_p), ctypes.POINTER(c_p), P_i64, P_i64, c_i,
                                  c_d, c_d, P_d, c_i, c_i, c_u, c_p]),
        "pe_split_open": (c_i, [c_p, c_i64, c_i64, c_i, P_d, c_i, c_i, c_p, ctypes.POINTER(c_p)]),
        "pe_split_sumsq": (c_i, [c_p, P_d]),
        "pe_split_set_norm": (c_i, [c_p, c_d]),
        "pe_split_gram": (c_i, [c_p, c_i, c_p, c_i64]),
        "pe_split_step": (c_i, [c_p, c_i, c_p, c_i64]),
        "pe_split_close": (c_i, [c_p]),
        "pe_polar_fast": (c_i, [c_p, c_i64, c_i64, P_d, c_i, c_i, c_i, c_p]),
        "pe_polar_fast_batched": (c_i, [ctypes.POINTER(c_p), P_i64, P_i64, c_i, P_d, c_i, c_i, c_d, c_d, c_i, c_u,
                                        c_p]),
        "pe_spectrum_bound": (c_i, [c_p, c_i64, c_i64, ctypes.POINTER(ctypes.c_float), c_i, P_d, P_d, c_p]),
        "pe_spectrum_aware_table": (c_i, [c_d, c_d, c_d, c_i, P_d, P_d]),
        "pe_spectrum_aware_table_ex": (c_i, [c_d, c_d, c_d, c_i, c_d, c_u, P_d, P_d]),
        "pe_polar_spectrum_aware": (c_i, [c_p, c_i64, c_i64, c_d, c_i, c_i, ctypes.POINTER(ctypes.c_float), c_i,
                                          P_d, c_p]),
        "pe_polar_spectrum_aware_ex": (c_i, [c_p, c_i64, c_i64, c_d, c_i, c_i, ctypes.POINTER(ctypes.c_float), c_i,
                                             c_d, c_u, P_d, c_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def declared_symbols() -> List[str]:
    """Entry points declared in include/polar_express.h."""
    import re
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+\**(pe_\w+)\s*\(", text, re.M)))


def _check(code: int):
    if code != PE_OK:
        msg = lib().pe_last_error().decode(errors="replace")
        raise PolarExpressError(code, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ offline stage

def pe_coeffs(degree: int, l: float, T: int, safety: float = 1.01, cushion: Optional[float] = None,
              skip_last: bool = False, return_info: bool = False):
    """Coefficient table (T, 3) float64; with return_info also the bounds
    (T+1, 2) and the Remez iteration count per step."""
    coeffs = np.zeros((T, 3), dtype=np.float64)
    bounds = np.zeros((T + 1, 2), dtype=np.float64)
    iters = (ctypes.c_int * max(T, 1))()
    flags = PE_SAFETY_SKIP_LAST if skip_last else 0
    code = lib().pe_coeffs_ex(int(degree), float(l), int(T), float(safety),
                              -1.0 if cushion is None else float(cushion), flags,
                              _dptr(coeffs), _dptr(bounds), iters)
    _check(code)
    if return_info:
        return coeffs, bounds, np.array(list(iters)[:T])
    return coeffs


# ------------------------------------------------------------- online stage

def _table(table) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 3))
    return t


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _io_of(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return PE_IO_FP32
    if t.dtype == torch.bfloat16:
        return PE_IO_BF16
    raise PolarExpressError(PE_EINVAL, f"unsupported tensor dtype {t.dtype}")


def _check_tensor(t):
    if not t.is_cuda:
        raise PolarExpressError(PE_EINVAL, "tensor must be on a CUDA device")
    if t.dim() != 2:
        raise PolarExpressError(PE_EINVAL, "tensor must be 2-D")
    if t.stride(1) != 1:
        raise PolarExpressError(PE_EINVAL, "tensor rows must be contiguous")


def pe_polar(X, table, dtype: str = "bf16", stream=None, norm_scale: float = 1.01,
             norm_eps: float = 1e-7):
    """Overwrite the 2-D CUDA tensor X (float32 or bfloat16) with the Polar
    Express approximation of polar(X). Asynchronous on ``stream``."""
    _check_tensor(X)
    tab = _table(table)
    code = lib().pe_polar_ex(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], X.stride(0), _io_of(X),
                             _dptr(tab), tab.shape[0], DTYPES[dtype], float(norm_scale), float(norm_eps),
                             ctypes.c_void_p(_stream_handle(stream)))
    _check(code)
    return X


def _fp32_matrix(X):
    import torch
    _check_tensor(X)
    if X.dtype != torch.float32 or not X.is_contiguous():
        raise PolarExpressError(PE_EINVAL, "X must be a contiguous float32 CUDA matrix")


def _start_vector(X, v0) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(v0, dtype=np.float32).reshape(-1))
    if v.shape[0] != min(X.shape[0], X.shape[1]):
        raise PolarExpressError(PE_EINVAL, "v0 must have min(m, n) entries")
    return v


_SA_KEYS = ("applied", "z", "f", "a", "b", "l_after")


def pe_spectrum_bound(X, v0, iters: int = 10, stream=None):
    """(z, f) of the spectrum-aware initialisation (App. H): z <= sigma_1 of
    the normalised X by ``iters`` power steps from the start vector v0
    (min(m, n) floats), f its Frobenius norm. Synchronises ``stream``."""
    _fp32_matrix(X)
    v = _start_vector(X, v0)
    z, f = ctypes.c_double(), ctypes.c_double()
    _check(lib().pe_spectrum_bound(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                                   v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(iters),
                                   ctypes.byref(z), ctypes.byref(f), ctypes.c_void_p(_stream_handle(stream))))
    return z.value, f.value


PE_SPECTRUM_GATE = 1


def pe_spectrum_aware_table(z: float, f: float, l: float, T: int, z_safety: float = 0.0, gate: bool = False):
    """(table (T + 1, 3), info) of the initialised iteration (host); the
    appendix's rule unless ``gate`` (PE_SPECTRUM_GATE) or ``z_safety``."""
    tab = np.zeros((T + 1, 3))
    info = np.zeros(6)
    _check(lib().pe_spectrum_aware_table_ex(float(z), float(f), float(l), int(T), float(z_safety),
                                            PE_SPECTRUM_GATE if gate else 0, _dptr(tab), _dptr(info)))
    d = dict(zip(_SA_KEYS, info.tolist()))
    d["applied"] = bool(d["applied"])
    return tab, d


def pe_polar_spectrum_aware(X, l: float, T: int, v0, dtype: str = "bf16", iters: int = 10, stream=None,
                            z_safety: Optional[float] = None, gate: bool = False):
    """In place on a contiguous float32 CUDA matrix: the App. H cubic (when it
    applies) and T Polar Express steps; returns the info dict. ``z_safety``
    None is the library's default for its FP32 bound (1e-5)."""
    _fp32_matrix(X)
    v = _start_vector(X, v0)
    info = np.zeros(6)
    args = (ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], float(l), int(T), DTYPES[dtype],
            v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(iters))
    if z_safety is None and not gate:
        _check(lib().pe_polar_spectrum_aware(*args, _dptr(info), ctypes.c_void_p(_stream_handle(stream))))
    else:
        _check(lib().pe_polar_spectrum_aware_ex(*args, float(1e-5 if z_safety is None else z_safety),
                                                PE_SPECTRUM_GATE if gate else 0, _dptr(info),
                                                ctypes.c_void_p(_stream_handle(stream))))
    d = dict(zip(_SA_KEYS, info.tolist()))
    d["applied"] = bool(d["applied"])
    return d


def pe_polar_batched(Xs: Sequence, table, dtype: str = "bf16", stream=None, flags: int = 0,
                     norm_scale: float = 1.01, norm_eps: float = 1e-7):
    """In place on a list of contiguous 2-D CUDA tensors of one dtype."""
    if len(Xs) == 0:
        return Xs
    io = _io_of(Xs[0])
    for t in Xs:
        _check_tensor(t)
        if not t.is_contiguous():
            raise PolarExpressError(PE_EINVAL, "batched tensors must be contiguous")
        if _io_of(t) != io:
            raise PolarExpressError(PE_EINVAL, "batched tensors must share one dtype")
    n = len(Xs)
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Xs])
    ms = (ctypes.c_int64 * n)(*[t.shape[0] for t in Xs])
    ns = (ctypes.c_int64 * n)(*[t.shape[1] for t in Xs])
    tab = _table(table)
    code = lib().pe_polar_batched_ex(ptrs, ms, ns, n, io, _dptr(tab), tab.shape[0], DTYPES[dtype],
                                     float(norm_scale), float(norm_eps), int(flags),
                                     ctypes.c_void_p(_stream_handle(stream)))
    _check(code)
    return Xs


def pe_polar_fast_batched(Xs: Sequence, table, restart: int = 3, dtype: str = "fp32", shift: float = 1e-3,
                          norm_eps: float = 1e-3, stream=None, flags: int = 0):
    """Alg. 4 (fast rectangular iteration) in place on a list of contiguous
    float32 CUDA matrices: blocks of ``restart`` steps, ``shift`` added to
    Y = X X^T in the first block, normalisation by 1.01 ||G||_F + norm_eps."""
    if len(Xs) == 0:
        return Xs
    for t in Xs:
        _fp32_matrix(t)
    n = len(Xs)
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Xs])
    ms = (ctypes.c_int64 * n)(*[t.shape[0] for t in Xs])
    ns = (ctypes.c_int64 * n)(*[t.shape[1] for t in Xs])
    tab = _table(table)
    _check(lib().pe_polar_fast_batched(ptrs, ms, ns, n, _dptr(tab), tab.shape[0], int(restart), float(shift),
                                       float(norm_eps), DTYPES[dtype], int(flags),
                                       ctypes.c_void_p(_stream_handle(stream))))
    return Xs


def pe_polar_fast(X, table, restart: int = 3, dtype: str = "fp32", stream=None):
    """Alg. 4 on one contiguous float32 CUDA matrix (shift and norm_eps 1e-3)."""
    _fp32_matrix(X)
    tab = _table(table)
    _check(lib().pe_polar_fast(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], _dptr(tab), tab.shape[0],
                               int(restart), DTYPES[dtype], ctypes.c_void_p(_stream_handle(stream))))
    return X


def pe_polar_batched_host(H_in: Sequence, H_out: Sequence, table, dtype: str = "bf16", ngroups: int = 0,
                          stream=None):
    """Host-buffer form: H_in / H_out are lists of contiguous float32 CPU
    tensors (pinned for asynchronous copies) of equal shapes per index. The
    copies are pipelined with the grouped compute on ``stream``."""
    n = len(H_in)
    if n == 0:
        return H_out
    if len(H_out) != n:
        raise PolarExpressError(PE_EINVAL, "H_in and H_out must have the same length")
    for a, b in zip(H_in, H_out):
        for t in (a, b):
            if t.is_cuda or t.dim() != 2 or not t.is_contiguous() or _io_of(t) != PE_IO_FP32:
                raise PolarExpressError(PE_EINVAL, "host matrices must be contiguous 2-D float32 CPU tensors")
        if a.shape != b.shape:
            raise PolarExpressError(PE_EINVAL, "H_in and H_out must have the same shapes")
    arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    ms = (ctypes.c_int64 * n)(*[t.shape[0] for t in H_in])
    ns = (ctypes.c_int64 * n)(*[t.shape[1] for t in H_in])
    tab = _table(table)
    _check(lib().pe_polar_batched_host(arr(H_in), arr(H_out), ms, ns, n, _dptr(tab), tab.shape[0], DTYPES[dtype],
                                       int(ngroups), ctypes.c_void_p(_stream_handle(stream))))
    return H_out


def pe_muon_batched(Ws: Sequence, Gs: Sequence, Ms: Sequence, beta: float, lr: float, table,
                    dtype: str = "bf16", stream=None, flags: int = 0):
    """Fused Muon update on lists of contiguous float32 CUDA tensors of equal
    shapes per index: M <- beta M + (1 - beta) G, W <- W - lr polar(M)."""
    n = len(Ws)
    if n == 0:
        return Ws
    if len(Gs) != n or len(Ms) != n:
        raise PolarExpressError(PE_EINVAL, "W, G and M lists must have the same length")
    for W, G, M in zip(Ws, Gs, Ms):
        for t in (W, G, M):
            _check_tensor(t)
            if not t.is_contiguous() or _io_of(t) != PE_IO_FP32:
                raise PolarExpressError(PE_EINVAL, "W, G, M must be contiguous float32 tensors")
        if not (W.shape == G.shape == M.shape):
            raise PolarExpressError(PE_EINVAL, "W, G and M must have the same shape")
    arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    ms = (ctypes.c_int64 * n)(*[t.shape[0] for t in Gs])
    ns = (ctypes.c_int64 * n)(*[t.shape[1] for t in Gs])
    tab = _table(table)
    _check(lib().pe_muon_batched(arr(Ws), arr(Gs), arr(Ms), ms, ns, n, float(beta), float(lr), _dptr(tab),
                                 tab.shape[0], DTYPES[dtype], int(flags), ctypes.c_void_p(_stream_handle(stream))))
    return Ws


def pe_sync_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status; raises
    PolarExpressError for a non-OK status."""
    code = lib().pe_sync_status(ctypes.c_void_p(_stream_handle(stream)))
    _check(code)
    return code


def pe_launch_count() -> int:
    return int(lib().pe_launch_count())


TRACE_KINDS = ["norm_partials", "prepare", "simt_gram", "simt_square", "simt_update", "umma_step",
               "umma_gram", "umma_square", "umma_update", "simt_gram_reduce", "fast_gemm", "fast_shift"]


def pe_trace_enable(on: bool = True):
    _check(lib().pe_trace_enable(1 if on else 0))


def pe_trace_read() -> dict:
    """{kernel kind: (launches, total ms)} for the traced launches."""
    n = len(TRACE_KINDS)
    cnt = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    _check(lib().pe_trace_read(cnt, ms, n))
    return {k: (int(cnt[i]), float(ms[i])) for i, k in enumerate(TRACE_KINDS) if cnt[i]}


def pe_release():
    lib().pe_release()


def pe_debug_set(key: int, value: int):
    _check(lib().pe_debug_set(int(key), int(value)))


def pe_version() -> int:
    return int(lib().pe_version())


# ------------------------------------------------------ long-side split

class Split:
    """One rank's block of a matrix split along its long side (pe_split_*).

    ``X``: the rank's block, a contiguous 2-D float32 CUDA tensor, in/out.
    ``short_is_rows``: True when the shared short side is X's rows (ranks
    hold column blocks), False when it is X's columns (ranks hold row
    blocks). The caller sums ``sumsq()`` and every ``gram`` result over the
    ranks; see shard.polar_split_long for the whole sequence."""

    def __init__(self, X, short_is_rows: bool, table, dtype: str = "bf16", stream=None):
        _check_tensor(X)
        if not X.is_contiguous() or _io_of(X) != PE_IO_FP32:
            raise PolarExpressError(PE_EINVAL, "the split block must be a contiguous float32 tensor")
        self.X = X
        self.table = _table(table)
        self.T = self.table.shape[0]
        self.s = X.shape[0] if short_is_rows else X.shape[1]
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(lib().pe_split_open(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], int(bool(short_is_rows)),
                                   _dptr(self.table), self.T, DTYPES[dtype], ctypes.c_void_p(self._stream),
                                   ctypes.byref(h)))
        self._h = h

    def sumsq(self) -> float:
        out = ctypes.c_double()
        _check(lib().pe_split_sumsq(self._h, ctypes.byref(out)))
        return out.value

    def set_norm(self, total_sumsq: float):
        _check(lib().pe_split_set_norm(self._h, float(total_sumsq)))

    def _a(self, A):
        _check_tensor(A)
        if _io_of(A) != PE_IO_FP32 or A.shape[0] < self.s or A.shape[1] < self.s:
            raise PolarExpressError(PE_EINVAL, "A must be a float32 CUDA tensor of at least s x s")
        return ctypes.c_void_p(A.data_ptr()), A.stride(0)

    def gram(self, t: int, A):
        p, lda = self._a(A)
        _check(lib().pe_split_gram(self._h, int(t), p, lda))

    def step(self, t: int, A):
        p, lda = self._a(A)
        _check(lib().pe_split_step(self._h, int(t), p, lda))

    def close(self):
        if self._h is not None and self._h.value:
            _check(lib().pe_split_close(self._h))
        self._h = None
