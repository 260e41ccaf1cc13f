"""pe_polar_noalloc: the allocation-free FP32 entry point.

Some callers cannot let the library call cudaMalloc: programs whose own
allocator owns all of device memory (a framework's caching pool, a server
with a fixed memory budget), loops that cannot take the synchronisation an
allocation can imply, and plug-in hosts that forbid a library's allocations.
pe_polar_noalloc serves them from a fixed device array inside the library.
These tests call it through the C ABI and compare it with pe_polar on the
FP32 path (within the FP32 bar of the other tests) and with the FP64
oracle, on calls in a row with different inputs and shapes, the largest
first: the array keeps the previous call's contents, so stale state from a
larger call would show up in the smaller ones.

This file is named to be collected last, so that a run that stops at its
first failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2505_16932_gb300 as pe
from paper_2505_16932_gb300 import build as B

FP32_TOL = 1e-5


def _lib():
    B.build()
    L = pe.lib()
    f = L.pe_polar_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                  ctypes.c_void_p]
    return L


def _call(L, X, table, stream):
    tab = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 3))
    return L.pe_polar_noalloc(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                              tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), tab.shape[0],
                              ctypes.c_void_p(stream))


def test_noalloc_rejects_oversized_matrix():
    """Sizes beyond the static workspace fail with a clear message before any
    device work (no GPU needed)."""
    L = _lib()
    tab = np.tile([1.875, -1.25, 0.375], (2, 1)).astype(np.float64)
    fake = ctypes.c_void_p(0x100000)
    r = L.pe_polar_noalloc(fake, 4096, 4096, tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, None)
    assert r == pe.PE_EINVAL
    msg = L.pe_last_error().decode()
    assert "workspace" in msg and "33554432" in msg
    assert L.pe_polar_noalloc(None, 8, 8, tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, None) == pe.PE_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_pe_polar_and_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    table = pe.pe_coeffs(5, 1e-3, 6, 1.01)
    rng = np.random.default_rng(2024)
    # calls in a row: the largest matrix first, then smaller ragged ones of
    # other shapes (tall, wide), then the first shape again with new entries
    for shape in ((768, 3072), (300, 129), (129, 520), (768, 3072)):
        G = rng.standard_normal(shape).astype(np.float32)
        ref = torch.from_numpy(G).cuda()
        pe.pe_polar(ref, table, "fp32")
        X = torch.from_numpy(G).cuda()
        assert _call(L, X, table, stream) == pe.PE_OK, L.pe_last_error().decode()
        torch.cuda.synchronize()
        got = X.cpu().numpy().astype(np.float64)
        want = ref.cpu().numpy().astype(np.float64)
        assert O.rel_fro(got, want) <= FP32_TOL, (shape, O.rel_fro(got, want))
        if shape[0] * shape[1] <= 300 * 520:   # the FP64 oracle on the small shapes
            fp64 = O.polar_express(G.astype(np.float64), table)
            assert O.rel_fro(got, fp64) <= FP32_TOL, (shape, O.rel_fro(got, fp64))
