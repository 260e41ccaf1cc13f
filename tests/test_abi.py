"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds, loads without a GPU driver, and exports every entry
  point that include/polar_express.h declares;
* pe_coeffs (C++ FP64 solver) reproduces the oracle's table bit for bit over
  a grid of degrees, lower bounds, step counts and safety settings;
* argument errors are reported synchronously with a message.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import paper_2505_16932_gb300 as pe
from paper_2505_16932_gb300 import build as B


@pytest.fixture(scope="module")
def L():
    B.build()
    return pe.lib()


def test_exports_every_declared_symbol(L):
    declared = pe.declared_symbols()
    assert "pe_coeffs" in declared and "pe_polar" in declared and "pe_polar_batched" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert pe.pe_version() >= 10000


GRID = [(d, l, T, s) for d in (3, 5)
        for l in (1e-7, 1e-5, 1e-4, 1e-3, 0.02407327424182761, 0.03, 0.1, 0.5, 1.0)
        for T in (1, 2, 5, 8, 12, 16)
        for s in (1.0, 1.01)]


@pytest.mark.parametrize("degree,l,T,safety", GRID)
def test_coeffs_bit_exact_vs_oracle(L, degree, l, T, safety):
    tab, bounds, iters = pe.pe_coeffs(degree, l, T, safety, return_info=True)
    rows, ob, info = O.optimal_composition(l, T, degree=degree, safety=safety, return_info=True)
    assert tab.tolist() == [list(r) for r in rows]
    assert bounds.tolist() == [list(b) for b in ob]


@pytest.mark.parametrize("cushion", [0.0, 0.1, 0.05])
def test_coeffs_cushion_and_skip_last(L, cushion):
    tab = pe.pe_coeffs(5, 1e-3, 6, 1.01, cushion=cushion, skip_last=True)
    rows, _ = O.optimal_composition(1e-3, 6, cushion=cushion, safety=1.01, safety_skip_last=True)
    assert tab.tolist() == [list(r) for r in rows]


def test_coeffs_remez_iterations(L):
    _, _, iters = pe.pe_coeffs(5, 1e-3, 10, 1.01, return_info=True)
    for t, it in enumerate(iters):
        assert 0 <= it <= 5
    assert iters[-1] == 0          # converged rows take the NS shortcut


@pytest.mark.parametrize("args", [(4, 1e-3, 5, 1.01), (5, 0.0, 5, 1.01), (5, 1.5, 5, 1.01),
                                  (5, 1e-3, 0, 1.01), (5, 1e-3, 65, 1.01), (5, 1e-3, 5, 0.9),
                                  (5, float("nan"), 5, 1.01)])
def test_coeffs_argument_errors(L, args):
    with pytest.raises(pe.PolarExpressError) as ei:
        pe.pe_coeffs(*args)
    assert ei.value.code == pe.PE_EINVAL
    assert L.pe_last_error().decode()


def test_coeffs_null_output(L):
    assert L.pe_coeffs(5, 1e-3, 5, 1.01, None, None) == pe.PE_EINVAL


def test_debug_key_errors(L):
    assert L.pe_debug_set(99, 0) == pe.PE_EINVAL


def test_polar_argument_errors_without_gpu(L):
    """Argument validation happens before any CUDA call, so it works here."""
    tab = np.ones((5, 3))
    P = ctypes.POINTER(ctypes.c_double)
    tp = tab.ctypes.data_as(P)
    # NULL matrix
    assert L.pe_polar(None, 4, 4, tp, 5, pe.PE_BF16, None) == pe.PE_EINVAL
    # bad sizes / T / dtype
    fake = ctypes.c_void_p(0x10000)
    assert L.pe_polar(fake, 0, 4, tp, 5, pe.PE_BF16, None) == pe.PE_EINVAL
    assert L.pe_polar(fake, 4, 4, tp, 0, pe.PE_BF16, None) == pe.PE_EINVAL
    assert L.pe_polar(fake, 4, 4, tp, 5, 7, None) == pe.PE_EINVAL
    assert L.pe_polar(fake, 4, 4, None, 5, pe.PE_BF16, None) == pe.PE_EINVAL
    bad = np.array([[1.0, float("inf"), 0.0]])
    assert L.pe_polar(fake, 4, 4, bad.ctypes.data_as(P), 1, pe.PE_BF16, None) == pe.PE_EINVAL
    assert L.pe_polar_ex(fake, 4, 4, 3, 0, tp, 5, 0, 1.01, 1e-7, None) == pe.PE_EINVAL   # ld < n
    assert L.pe_polar_ex(fake, 4, 4, 4, 0, tp, 5, 0, -1.0, 1e-7, None) == pe.PE_EINVAL  # scale
    ptrs = (ctypes.c_void_p * 1)(None)
    ms = (ctypes.c_int64 * 1)(4)
    assert L.pe_polar_batched(ptrs, ms, ms, 1, tp, 5, pe.PE_BF16, None) == pe.PE_EINVAL
    assert L.pe_polar_batched(ptrs, ms, ms, 0, tp, 5, pe.PE_BF16, None) == pe.PE_EINVAL


def test_split_argument_errors_without_gpu(L):
    """pe_split_* validate their arguments before any CUDA call."""
    tab = np.ones((5, 3))
    P = ctypes.POINTER(ctypes.c_double)
    tp = tab.ctypes.data_as(P)
    fake = ctypes.c_void_p(0x10000)
    h = ctypes.c_void_p()
    assert L.pe_split_open(None, 4, 8, 1, tp, 5, pe.PE_BF16, None, ctypes.byref(h)) == pe.PE_EINVAL
    assert L.pe_split_open(fake, 4, 8, 1, tp, 5, pe.PE_BF16X3, None, ctypes.byref(h)) == pe.PE_EUNSUPPORTED
    assert L.pe_split_open(fake, 4, 8, 1, tp, 5, 7, None, ctypes.byref(h)) == pe.PE_EINVAL
    assert L.pe_split_open(fake, 0, 8, 1, tp, 5, pe.PE_BF16, None, ctypes.byref(h)) == pe.PE_EINVAL
    assert L.pe_split_open(fake, 4, 8, 1, tp, 0, pe.PE_BF16, None, ctypes.byref(h)) == pe.PE_EINVAL
    assert L.pe_split_open(fake, 4, 8, 1, tp, 5, pe.PE_BF16, None, None) == pe.PE_EINVAL
    assert h.value is None
    d = ctypes.c_double()
    assert L.pe_split_sumsq(None, ctypes.byref(d)) == pe.PE_EINVAL
    assert L.pe_split_set_norm(None, 1.0) == pe.PE_EINVAL
    assert L.pe_split_gram(None, 0, fake, 4) == pe.PE_EINVAL
    assert L.pe_split_step(None, 0, fake, 4) == pe.PE_EINVAL
    assert L.pe_split_close(None) == pe.PE_EINVAL


def test_host_entry_argument_errors_without_gpu(L):
    tab = np.ones((5, 3))
    P = ctypes.POINTER(ctypes.c_double)
    tp = tab.ctypes.data_as(P)
    ms = (ctypes.c_int64 * 1)(4)
    ptrs = (ctypes.c_void_p * 1)(None)
    assert L.pe_polar_batched_host(None, None, ms, ms, 1, tp, 5, pe.PE_BF16, 0, None) == pe.PE_EINVAL
    assert L.pe_polar_batched_host(ptrs, ptrs, ms, ms, 1, tp, 5, pe.PE_BF16, 0, None) == pe.PE_EINVAL
    assert L.pe_polar_batched_host(ptrs, ptrs, ms, ms, 0, tp, 5, pe.PE_BF16, 0, None) == pe.PE_EINVAL
    fake = (ctypes.c_void_p * 1)(0x10000)
    assert L.pe_polar_batched_host(fake, fake, ms, ms, 1, tp, 5, pe.PE_BF16, -1, None) == pe.PE_EINVAL


def test_spectrum_entry_argument_errors_without_gpu(L):
    F = ctypes.POINTER(ctypes.c_float)
    v = np.ones(4, dtype=np.float32)
    vz = np.zeros(4, dtype=np.float32)
    z, f = ctypes.c_double(), ctypes.c_double()
    fake = ctypes.c_void_p(0x10000)
    args = lambda X, m, n, vv, it: (X, m, n, vv.ctypes.data_as(F), it, ctypes.byref(z), ctypes.byref(f), None)  # noqa: E731
    assert L.pe_spectrum_bound(*args(None, 4, 8, v, 5)) == pe.PE_EINVAL
    assert L.pe_spectrum_bound(*args(fake, 0, 8, v, 5)) == pe.PE_EINVAL
    assert L.pe_spectrum_bound(*args(fake, 4, 8, v, -1)) == pe.PE_EINVAL
    assert L.pe_spectrum_bound(*args(fake, 4, 8, vz, 5)) == pe.PE_EINVAL
    assert b"nonzero" in L.pe_last_error()
    assert L.pe_spectrum_bound(*args(ctypes.c_void_p(0x10002), 4, 8, v, 5)) == pe.PE_EINVAL
    info = np.zeros(6)
    P = ctypes.POINTER(ctypes.c_double)
    assert L.pe_polar_spectrum_aware(fake, 4, 8, 1e-3, 5, 7, v.ctypes.data_as(F), 5, info.ctypes.data_as(P),
                                     None) == pe.PE_EINVAL
    assert L.pe_polar_spectrum_aware(fake, 4, 8, 0.0, 5, pe.PE_BF16, v.ctypes.data_as(F), 5,
                                     info.ctypes.data_as(P), None) == pe.PE_EINVAL
    tab = np.zeros((6, 3))
    assert L.pe_spectrum_aware_table(0.9, 1.0, 1e-3, -1, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_spectrum_aware_table(0.9, 1.0, 2.0, 5, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_spectrum_aware_table(float("nan"), 1.0, 1e-3, 5, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_spectrum_aware_table_ex(0.9, 1.0, 1e-3, 5, 1.0, 0, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_spectrum_aware_table_ex(0.9, 1.0, 1e-3, 5, -1e-3, 0, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_spectrum_aware_table_ex(0.9, 1.0, 1e-3, 5, 0.0, 2, tab.ctypes.data_as(P), None) == pe.PE_EINVAL
    assert L.pe_polar_spectrum_aware_ex(fake, 4, 8, 1e-3, 5, pe.PE_BF16, v.ctypes.data_as(F), 5, 0.0, 4,
                                        info.ctypes.data_as(P), None) == pe.PE_EINVAL


@pytest.mark.parametrize("z_safety,gate", [(0.0, False), (1e-5, False), (0.0, True), (1e-5, True)])
@pytest.mark.parametrize("z,f,l,T", [(0.95, 0.99, 1e-3, 5), (0.999, 0.99999, 1e-7, 8), (0.72, 1.0, 1e-4, 3),
                                     (0.5, 0.99, 1e-3, 5), (0.7, 0.99, 1e-3, 4), (0.9, 1.0, 1e-3, 0),
                                     (0.0, 0.0, 1e-3, 5), (0.8, 1.0, 1e-4, 4)])
def test_spectrum_aware_table_matches_oracle(L, z, f, l, T, z_safety, gate):
    """Host table of the App. H initialisation against the oracle's, with the
    appendix's rule and with each option: the cubic row to rounding, the
    following composition from the same l'."""
    from oracle import spectrum_init as S
    tab, info = pe.pe_spectrum_aware_table(z, f, l, T, z_safety=z_safety, gate=gate)
    ref, rinfo = S.spectrum_aware_table(z, f, l, T, z_safety=z_safety, gate=gate)
    assert info["applied"] == rinfo["applied"]
    assert tab.shape == (T + 1, 3) and len(ref) == T + 1
    assert np.allclose(tab, np.array(ref), rtol=1e-12, atol=0)
    assert math.isclose(info["l_after"], rinfo["l_after"], rel_tol=1e-14)
    if info["applied"]:
        assert tab[0, 2] == 0.0
        assert math.isclose(info["a"], rinfo["a"], rel_tol=1e-14) and math.isclose(info["b"], rinfo["b"], rel_tol=1e-14)
