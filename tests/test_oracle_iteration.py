"""Pins for the oracle's online stage, truth and error metrics.

The FP64 matrix iteration is checked against its spectral form
U p(x) V^T (App. C: p(M) acts on the singular values), which fixes the
orientation of A = X X^T, the combination b A + c A^2 and the update
a X + B X independently of the code under test; polar via SVD is checked
against its definition (orthogonal factor, symmetric PSD cofactor), the 2x2
closed form, vectors, orthogonal inputs and brute-force convergence.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def _table(l, T, safety=1.01):
    rows, _ = O.optimal_composition(l, T, safety=safety)
    return rows


@pytest.mark.parametrize("m,n", [(40, 24), (24, 40), (33, 33), (1, 7), (7, 1), (64, 200)])
def test_matrix_iteration_equals_spectral_form(m, n):
    case = synth.random_svd_case(seed=m * 100 + n, m=m, n=n, lo=1e-2, hi=1.0)
    tab = _table(1e-3, 6)
    X = O.polar_express(case.G, tab)
    Y = O.polar_express_spectral(case.U, case.s, case.V, tab)
    assert X.shape == (m, n)
    assert np.linalg.norm(X - Y) <= 1e-12 * max(1.0, np.linalg.norm(Y))


def test_spectral_sampled_entries():
    case = synth.random_svd_case(seed=5, m=50, n=30)
    tab = _table(1e-3, 5)
    full = O.polar_express_spectral(case.U, case.s, case.V, tab)
    rng = np.random.default_rng(0)
    r = rng.integers(0, 50, 100)
    c = rng.integers(0, 30, 100)
    samp = O.polar_express_spectral(case.U, case.s, case.V, tab, rows=r, cols=c)
    assert np.allclose(samp, full[r, c], rtol=0, atol=1e-14)


def test_steps_match_paper_operands():
    """One step written with the paper's operand order (Sec. 3.5 Horner form
    X (aI + Y (bI + cY)), Y = X^T X on the tall side) equals the oracle's short
    side form (aI + (bA + cA^2)) X with A = X X^T, transposed."""
    rng = np.random.default_rng(3)
    G = rng.standard_normal((30, 12))  # tall: the oracle transposes to 12 x 30
    a, b, c = 3.0, -2.5, 0.6
    X0 = G / (1.01 * np.linalg.norm(G) + 1e-7)
    Y = X0.T @ X0
    ref = X0 @ (a * np.eye(12) + Y @ (b * np.eye(12) + c * Y))
    got = O.polar_express(G, [(a, b, c)])
    assert np.allclose(got, ref, rtol=0, atol=1e-14)


def test_normalise():
    rng = np.random.default_rng(1)
    G = rng.standard_normal((9, 4))
    X, tr = O.normalise(G)
    assert tr and X.shape == (4, 9)
    nu = np.linalg.norm(G)
    assert abs(np.linalg.norm(X) - nu / (1.01 * nu + 1e-7)) < 1e-15
    X2, tr2 = O.normalise(G.T)
    assert not tr2 and np.array_equal(X2, X)
    X3, _ = O.normalise(G, scale=1.0, eps=1e-2)   # Alg. 1 variant
    assert abs(np.linalg.norm(X3) - nu / (nu + 1e-2)) < 1e-15


# ------------------------------------------------------------- polar(G)

@pytest.mark.parametrize("m,n", [(5, 5), (8, 3), (3, 8), (17, 17), (30, 11)])
def test_polar_svd_definition(m, n):
    """polar(G) = Q with Q semi-orthogonal and G = Q H, H symmetric PSD
    (tall), or G = H Q (wide)."""
    rng = np.random.default_rng(m * 7 + n)
    G = rng.standard_normal((m, n))
    Q = O.polar_svd(G)
    k = min(m, n)
    if m >= n:
        assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-13)
        H = Q.T @ G
    else:
        assert np.allclose(Q @ Q.T, np.eye(k), atol=1e-13)
        H = G @ Q.T
    assert np.allclose(H, H.T, atol=1e-12)
    assert np.min(np.linalg.eigvalsh(0.5 * (H + H.T))) >= -1e-12


def test_polar_2x2_closed_form():
    rng = np.random.default_rng(2)
    for _ in range(100):
        M = rng.standard_normal((2, 2))
        assert np.allclose(O.polar_2x2(M), O.polar_svd(M), atol=1e-12)
    R = np.array([[0.0, -2.0], [2.0, 0.0]])   # 2 x rotation
    assert np.allclose(O.polar_2x2(R), R / 2)


def test_polar_of_orthogonal_is_itself():
    rng = np.random.default_rng(4)
    Q = synth.haar_orthonormal(rng, 12, 12)
    S = synth.haar_orthonormal(rng, 20, 6)
    for A in (Q, S, S.T):
        assert np.allclose(O.polar_svd(A), A, atol=1e-13)
        # all normalised singular values equal 1/(1.01 sqrt(k)); converge from there
        k = min(A.shape)
        l = 1.0 / (1.02 * math.sqrt(k))
        X = O.polar_express(A, _table(l, 10, safety=1.0))
        assert np.allclose(X, A, atol=1e-13)


def test_vector_case():
    v = np.array([[3.0], [4.0], [0.0]])
    assert np.allclose(O.polar_svd(v), v / 5)
    X = O.polar_express(v, _table(0.9, 6, safety=1.0))
    assert np.allclose(X, v / 5, atol=1e-14)
    X = O.polar_express(v.T, _table(0.9, 6, safety=1.0))
    assert np.allclose(X, v.T / 5, atol=1e-14)


@pytest.mark.parametrize("m", range(1, 9))
def test_bruteforce_tiny_converges_to_svd_polar(m):
    rng = np.random.default_rng(100 + m)
    for n in range(1, 9):
        G = rng.standard_normal((m, n))
        sv = np.linalg.svd(G, compute_uv=False)
        if sv.min() < 1e-3 * sv.max():
            continue
        l = 0.5 * sv.min() / (1.01 * np.linalg.norm(G))
        X = O.polar_express(G, _table(l, 14, safety=1.0))
        assert np.allclose(X, O.polar_svd(G), atol=1e-12), (m, n)


def test_fp64_iteration_meets_greedy_error_bound():
    """Eq. error: with sigma(X0) inside [l, 1], ||polar - X_T||_2 <= 1 - l_{T+1}."""
    case = synth.random_svd_case(seed=9, m=60, n=40, lo=1e-2, hi=1.0)
    x = case.s / (1.01 * np.linalg.norm(case.s) + 1e-7)
    l = float(x.min())
    rows, bounds = O.optimal_composition(l, 4)
    X = O.polar_express(case.G, rows)
    err2 = np.linalg.norm(X - case.U @ case.V.T, 2)
    assert err2 <= 1 - bounds[-1][0] + 1e-12


# -------------------------------------------------------------- metrics

def test_error_metrics():
    rng = np.random.default_rng(6)
    Q = synth.haar_orthonormal(rng, 10, 6)
    assert O.max_sigma_err(Q) < 1e-14
    assert abs(O.max_sigma_err(0.5 * Q) - 0.5) < 1e-14
    assert abs(O.err_polar_fro(0.5 * Q, Q) - 0.5) < 1e-14
    assert abs(O.rel_fro(2 * Q, Q) - 1.0) < 1e-14


def test_restricted_errors():
    case = synth.random_svd_case(seed=8, m=30, n=20, lo=1e-6, hi=1.0)
    P = case.U @ case.V.T
    fro, mx = O.restricted_errors(P, case.U, case.s, case.V, gamma=1e-3)
    assert fro < 1e-13 and mx < 1e-13
    keep = case.s >= 1e-3
    f = np.where(keep, 1.0, 0.0)          # truncated polar factor (App. H.1)
    Pt = (case.U * f) @ case.V.T
    fro, mx = O.restricted_errors(Pt, case.U, case.s, case.V, gamma=1e-3)
    assert fro < 1e-13 and mx < 1e-13
    fro, mx = O.restricted_errors(0.9 * P, case.U, case.s, case.V)
    assert abs(mx - 0.1) < 1e-12
