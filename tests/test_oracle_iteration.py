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


# ----------------------------------------- Alg. 4 (fast rectangular iteration)

@pytest.mark.parametrize("m,n", [(40, 170), (170, 40), (32, 32)])
def test_fast_rectangular_restart_one_is_the_baseline(m, n):
    """Restarting after every step is the baseline method (appendix on
    rectangular matrices): same normalisation, no shift."""
    G = np.random.default_rng(m * n).standard_normal((m, n))
    tab, _ = O.optimal_composition(1e-3, 6, safety=1.01)
    ref = O.polar_express(G, tab, scale=1.01, eps=1e-3)
    got = O.fast_rectangular(G, tab, restart=1, shift=0.0)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("restart", [2, 3, 6])
def test_fast_rectangular_without_shift_equals_the_baseline(restart):
    """Without the shift, X_T = Q_T X_0 = (p_T o ... o p_1)(X_0) (the induction
    of the appendix): any restart interval gives the baseline's result up to
    FP64 rounding on a well-conditioned input."""
    case = synth.random_svd_case(seed=7, m=48, n=200, lo=0.1)
    tab, _ = O.optimal_composition(1e-1, 6, safety=1.01)
    ref = O.polar_express(case.G, tab, scale=1.01, eps=1e-3)
    got = O.fast_rectangular(case.G, tab, restart=restart, shift=0.0)
    assert np.max(np.abs(got - ref)) <= 1e-10


@pytest.mark.parametrize("restart,shift", [(3, 1e-3), (2, 1e-3), (6, 1e-2)])
@pytest.mark.parametrize("m,n", [(40, 160), (160, 40)])
def test_fast_rectangular_matches_its_spectral_form(restart, shift, m, n):
    """Matrix recursion (Y, Q, R) against the scalar recursion on the
    singular values, q <- q h(y q^2), with the shift only in the first block."""
    case = synth.random_svd_case(seed=m + n + restart, m=m, n=n, lo=1e-3)
    tab, _ = O.optimal_composition(1e-3, 6, safety=1.01)
    got = O.fast_rectangular(case.G, tab, restart=restart, shift=shift)
    ref = O.fast_rectangular_spectral(case.U, case.s, case.V, tab, restart=restart, shift=shift)
    assert np.max(np.abs(got - ref)) <= 1e-10


def test_fast_rectangular_shift_only_in_first_block():
    """The shift changes the first block only: the later blocks are the plain
    iteration applied to the first block's output."""
    case = synth.random_svd_case(seed=3, m=30, n=120, lo=1e-2)
    tab, _ = O.optimal_composition(1e-2, 6, safety=1.01)
    full, blocks = O.fast_rectangular(case.G, tab, restart=3, return_blocks=True)
    X3 = blocks[0]
    # the remaining 3 steps without shift, on X3 as already normalised (scale 1, eps 0)
    X = X3.copy()
    for (a, b, c) in tab[3:]:
        A = X @ X.T
        X = a * X + (b * A + c * (A @ A)) @ X
    assert np.max(np.abs(full - X)) <= 1e-10
    # and the first block differs from the unshifted one
    noshift = O.fast_rectangular(case.G, tab[:3], restart=3, shift=0.0)
    assert np.max(np.abs(noshift - X3)) > 1e-4


def test_fast_rectangular_still_converges_to_polar():
    """With the shift the early output differs, yet the restarted iteration
    still converges to polar(G) (the appendix's remark): 4 blocks of 3."""
    case = synth.random_svd_case(seed=5, m=32, n=128, lo=1e-2)
    tab, _ = O.optimal_composition(1e-2, 12, safety=1.01)
    got = O.fast_rectangular(case.G, tab, restart=3)
    P = (case.U @ case.V.T)
    assert O.err_polar_fro(got, P) <= 1e-6
    assert O.max_sigma_err(got) <= 1e-6
