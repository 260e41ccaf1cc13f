"""Pins of the spectrum-aware initialisation oracle (App. H, k = 1).

Each pin checks the oracle against something other than itself: the two
interpolation conditions of Eq. init_poly, the 2 x 2 linear system they
define (solved by LAPACK), the paper's claims p(1) > 1/sqrt(2) and
p(x) >= x / w on [0, w], the Rayleigh-quotient bound z <= sigma_1 against
the SVD, the matrix step against the scalar map on known singular values, and
the convergence benefit the appendix reports on the 32 x 32 matrix with
sigma_j = j^-5 (its figure on the spectrum-aware scheme).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import spectrum_init as S


def _haar(rng, n):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("z", [0.7072, 0.75, 0.8, 0.9, 0.99, 0.999999])
def test_cubic_interpolates_both_ends(z):
    a, b = S.init_cubic_unit(z)
    w = math.sqrt(1 - z * z)
    assert abs(a * w + b * w ** 3 - 1) <= 1e-12
    assert abs(a * z + b * z ** 3 - 1) <= 1e-12
    # the same (a, b) from the 2 x 2 system p(w) = p(z) = 1 (LAPACK)
    sol = np.linalg.solve(np.array([[w, w ** 3], [z, z ** 3]]), np.ones(2))
    assert np.allclose(sol, [a, b], rtol=1e-9, atol=0)


def test_paper_claims_on_the_cubic():
    """p(1) > 1/sqrt(2) for every admissible z, p above the chord x / w on
    [0, w], p decreasing on [z, 1] and at most 1 on [0, w] and [z, 1]."""
    for z in np.linspace(1 / math.sqrt(2) + 1e-4, 1 - 1e-6, 400):
        a, b = S.init_cubic_unit(z)
        w = math.sqrt(1 - z * z)
        p = lambda x: a * x + b * x ** 3  # noqa: E731
        assert p(1.0) > 1 / math.sqrt(2)
        x = np.linspace(0, w, 201)
        assert np.all(p(x) >= x / w - 1e-12)
        assert np.all(p(x) <= 1 + 1e-12)
        y = np.linspace(z, 1, 201)
        assert np.all(np.diff(p(y)) <= 1e-15)
        assert np.all(p(y) <= 1 + 1e-12)


def test_general_norm_is_the_unit_cubic_of_x_over_f():
    for f in (0.5, 0.99, 2.0):
        for zn in (0.72, 0.9, 0.995):
            a, b, w = S.init_cubic(zn * f, f)
            a1, b1 = S.init_cubic_unit(zn)
            for x in (0.1, 0.5, 0.8, 1.0):
                assert abs((a * x * f + b * (x * f) ** 3) - (a1 * x + b1 * x ** 3)) <= 1e-12
            assert abs(w - f * math.sqrt(1 - zn * zn)) <= 1e-15 * f
    assert S.init_cubic(0.7, 1.0) is None          # 2 z^2 <= f^2: the intervals overlap
    assert S.init_cubic(1.0, 1.0) is None          # w = 0
    assert S.init_cubic(0.0, 0.0) is None


def test_power_bound_is_a_lower_bound_and_converges():
    rng = np.random.default_rng(3)
    for m, n in ((20, 30), (30, 20), (17, 17)):
        X = rng.standard_normal((m, n))
        s1 = np.linalg.svd(X, compute_uv=False)[0]
        v0 = rng.standard_normal(n)
        prev = 0.0
        for it in range(0, 12):
            z = S.power_bound(X, v0, it)
            assert z <= s1 * (1 + 1e-14)
            assert z >= prev * (1 - 1e-12)          # monotone for the power method
            prev = z
    # gapped spectrum: the bound is tight after a few steps
    U, V = _haar(rng, 24), _haar(rng, 24)
    s = np.concatenate([[1.0], np.linspace(0.2, 0.01, 23)])
    X = (U * s) @ V.T
    z = S.power_bound(X, rng.standard_normal(24), 8)
    assert 1.0 - 1e-9 <= z <= 1.0 + 1e-14


def test_cubic_step_is_the_scalar_map_on_singular_values():
    rng = np.random.default_rng(4)
    n = 24
    U, V = _haar(rng, n), _haar(rng, n)
    s = np.concatenate([[1.0], np.geomspace(0.3, 1e-4, n - 1)])
    G = (U * s) @ V.T
    X0, _ = O.normalise(G)
    f = float(np.linalg.norm(X0))
    z = S.power_bound(X0.T, rng.standard_normal(n), 10)
    a, b, w = S.init_cubic(z, f)
    X = O.polar_express(G, [(a, b, 0.0)])
    x = s / (1.01 * np.linalg.norm(s) + 1e-7)
    ref = (U * (a * x + b * x ** 3)) @ V.T
    assert np.max(np.abs(X - ref)) <= 1e-13
    # the mapped spectrum: at most 1, and each value at least min(x / w, p(f))
    px = a * x + b * x ** 3
    pf = a * f + b * f ** 3
    assert px.max() <= 1 + 1e-12
    assert np.all(px >= np.minimum(x / w, pf) * (1 - 1e-12))


def _spectra(tail):
    k = 768
    s = 1.0 / np.arange(1, k + 1) if tail is None else np.concatenate([[1.0], np.geomspace(*tail, k - 1)])
    x = s / (1.01 * np.linalg.norm(s) + 1e-7)
    return x, float(np.linalg.norm(x)), float(x.max())


def _forced(z, f, l, T):
    a, b, w = S.init_cubic(z, f)
    rest = O.optimal_composition(min(l / w, a * f + b * f ** 3), T, safety=1.01)[0]
    return [(a, b, 0.0)] + [tuple(r) for r in rest]


@pytest.mark.parametrize("tail", [None, (0.01, 1e-4)])
def test_paper_rule_applies_the_cubic_whenever_the_intervals_are_disjoint(tail):
    """The appendix builds the cubic whenever [0, w] and [z, f] are disjoint:
    the table is the cubic followed by the composition for [l', 1], without
    any further condition, whatever it does to the final error."""
    x, f, z = _spectra(tail)
    assert 2 * z * z > f * f
    table, info = S.spectrum_aware_table(z, f, 1e-4, 4)
    assert info["applied"] and info["z"] == z
    assert np.array_equal(np.array(table), np.array(_forced(z, f, 1e-4, 4)))
    # the z shrink option moves z, and only z
    table2, info2 = S.spectrum_aware_table(z, f, 1e-4, 4, z_safety=1e-5)
    assert info2["z"] == z * (1 - 1e-5)
    assert np.array_equal(np.array(table2), np.array(_forced(z * (1 - 1e-5), f, 1e-4, 4)))


def test_gate_keeps_the_cubic_only_when_its_final_bound_is_better():
    """The gate option (not the appendix's rule). Spectra 1/i (the GPT-2-like
    workload): the intervals are disjoint but the tail gains only f / w ~ 1.6,
    less than a quintic step, so the gate keeps the plain composition, and it
    is indeed the more accurate one; a gap of 100 (sigma_2 = 0.01) keeps the
    cubic, which is then the more accurate."""
    for tail, keep in ((None, False), ((0.01, 1e-4), True)):
        x, f, z = _spectra(tail)
        table, info = S.spectrum_aware_table(z, f, 1e-4, 4, gate=True)
        assert info["applied"] == keep
        plain, _ = O.optimal_composition(1e-4, 5, safety=1.01)
        forced = _forced(z, f, 1e-4, 4)
        e_plain = np.max(np.abs(O.compose_scalar(x, plain) - 1))
        e_forced = np.max(np.abs(O.compose_scalar(x, forced) - 1))
        assert (e_forced < e_plain) == keep, (e_forced, e_plain)
        assert np.allclose(np.array(table), np.array(forced if keep else plain), rtol=0, atol=0)


def test_no_cubic_without_a_dominant_singular_value():
    rng = np.random.default_rng(5)
    G = rng.standard_normal((16, 40))               # flat spectrum: z far below f / sqrt 2
    X, table, info = S.spectrum_aware_polar(G, 1e-3, 5, rng.standard_normal(16), 10)
    assert not info["applied"] and len(table) == 6
    ref, _ = O.optimal_composition(1e-3, 6, safety=1.01)
    assert np.allclose(np.array(table), np.array(ref), rtol=0, atol=0)


def test_power_law_spectrum_converges_faster_with_the_cubic():
    """32 x 32, sigma_j = j^-5 (the appendix's example): counting the cubic as
    an iteration, the initialised iteration is far closer to U V^T than plain
    Polar Express at the same total step count once either gets close."""
    rng = np.random.default_rng(0)
    n = 32
    U, V = _haar(rng, n), _haar(rng, n)
    s = np.arange(1, n + 1, dtype=np.float64) ** -5.0
    G = (U * s) @ V.T
    P = U @ V.T
    l = s[-1] / (1.01 * np.linalg.norm(s))
    v0 = rng.standard_normal(n)
    for K, gain in ((11, 3.0), (12, 20.0), (13, 1e3)):
        plain, _ = O.optimal_composition(l, K, safety=1.01)
        e_plain = np.linalg.norm(O.polar_express(G, plain) - P, 2)
        X, table, info = S.spectrum_aware_polar(G, l, K - 1, v0, 10)
        assert info["applied"] and len(table) == K
        e_init = np.linalg.norm(X - P, 2)
        assert e_init * gain < e_plain, (K, e_init, e_plain)
