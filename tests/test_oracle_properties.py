"""Property-based pins of the oracle (hypothesis; skipped where it is not
installed): on random intervals the Remez quintic equioscillates and no grid
point beats it, the greedy composition maps [l, 1] into its bounds, and on
random small matrices the FP64 iteration equals the scalar map on the singular
values (App. C) and the C-ABI coefficient solver reproduces the oracle's
table bit for bit.
"""
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402


def _p(row, x):
    a, b, c = row
    return a * x + b * x ** 3 + c * x ** 5


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(st.floats(min_value=-7.0, max_value=-0.05), st.floats(min_value=0.0, max_value=0.5))
def test_remez_equioscillates_on_random_intervals(log_l, log_du):
    u = 10.0 ** log_du
    l = u * 10.0 ** log_l
    a, b, c, info = O.optimal_quintic(l, u, return_info=True)
    if info["shortcut"]:
        return
    E = info["E"]
    for x, s in zip([l, info["x1"], info["x2"], u], [1, -1, 1, -1]):
        assert abs((1 - _p((a, b, c), x)) - s * E) <= 1e-13 * max(1.0, abs(a) * u)
    g = np.linspace(l, u, 20001)
    assert np.max(np.abs(1 - _p((a, b, c), g))) <= abs(E) + 1e-12


@settings(max_examples=25, deadline=None, derandomize=True, database=None)
@given(st.floats(min_value=-7.0, max_value=-0.5), st.integers(min_value=1, max_value=10))
def test_composition_maps_interval_into_bounds(log_l, T):
    l = 10.0 ** log_l
    rows, bounds = O.optimal_composition(l, T)
    x = np.geomspace(l, 1.0, 4001)
    y = O.compose_scalar(x, rows)
    lo, hi = bounds[-1]
    # near x = 1 each step's rounding is amplified by the later steps' slopes at
    # u_t: tolerance 8 eps sum_t prod_{s>=t} max(1, |p_s'(u_s)|)
    amp, tot = 1.0, 0.0
    for t in range(T - 1, -1, -1):
        a, b, c = rows[t]
        u = bounds[t][1]
        amp *= max(1.0, abs(a + 3 * b * u * u + 5 * c * u ** 4))
        tot += amp
    eps = np.finfo(np.float64).eps
    assert y.min() >= lo - 1e-12 and y.max() <= hi + 8 * eps * tot + 1e-12


@settings(max_examples=25, deadline=None, derandomize=True, database=None)
@given(st.integers(min_value=1, max_value=9), st.integers(min_value=1, max_value=9),
       st.integers(min_value=0, max_value=2 ** 31 - 1))
def test_iteration_is_the_scalar_map(m, n, seed):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    qu, _ = np.linalg.qr(rng.standard_normal((m, k)))
    qv, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s = np.sort(rng.uniform(0.01, 1.0, k))[::-1]
    G = (qu * s) @ qv.T
    rows, _ = O.optimal_composition(1e-2, 4, safety=1.01)
    got = O.polar_express(G, rows)
    ref = O.polar_express_spectral(qu, s, qv, rows)
    assert np.max(np.abs(got - ref)) <= 1e-12


@settings(max_examples=30, deadline=None, derandomize=True, database=None)
@given(st.floats(min_value=-7.0, max_value=0.0), st.integers(min_value=1, max_value=12),
       st.sampled_from([3, 5]), st.sampled_from([1.0, 1.01]))
def test_c_solver_bit_exact_on_random_inputs(log_l, T, degree, safety):
    import paper_2505_16932_gb300 as pe
    from paper_2505_16932_gb300 import build as B
    B.build()
    l = 10.0 ** log_l
    ref, _ = O.optimal_composition(l, T, degree=degree, safety=safety)
    got = pe.pe_coeffs(degree, l, T, safety)
    assert np.array_equal(np.asarray(got), np.asarray(ref, dtype=np.float64)), (l, T, degree, safety)
    assert not any(math.isnan(v) for row in ref for v in row)
