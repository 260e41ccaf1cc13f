"""Pins for the oracle's offline stage (coefficient solve).

Each test checks the oracle against something other than itself: the table
the paper prints, the equioscillation characterisation of the minimax
polynomial (Lemma in App. D), an LP solve of the same minimax problem on a
grid, the degree-3 closed form, the l/u -> 1 limit, the greedy bounds and
optimality of Thm. 1, the convergence bound of Thm. 2, and scalar facts the
paper states (App. F, App. G).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import minimax as MM

from conftest import read_golden

EPS = np.finfo(np.float64).eps


def p_eval(row, x):
    a, b, c = row
    x = np.asarray(x, dtype=np.float64)
    return a * x + b * x ** 3 + c * x ** 5


def dp_eval(row, x):
    a, b, c = row
    return a + 3 * b * x ** 2 + 5 * c * x ** 4


def dense_grid(l, u, n=200001):
    return np.linspace(l, u, n)


# ---------------------------------------------------------------- 4x4 solve

def test_gepp_matches_lapack():
    rng = np.random.default_rng(0)
    for _ in range(200):
        M = rng.standard_normal((4, 4))
        y = rng.standard_normal(4)
        z = np.array(O.gepp_solve(M.tolist(), y.tolist()))
        ref = np.linalg.solve(M, y)
        assert np.linalg.norm(z - ref) <= 64 * EPS * np.linalg.cond(M) * np.linalg.norm(ref)


def test_gepp_pivots():
    # zero leading entry forces a row swap; exact answer known
    M = [[0.0, 1.0], [2.0, 0.0]]
    assert O.gepp_solve(M, [3.0, 4.0]) == [2.0, 3.0]
    with pytest.raises(ZeroDivisionError):
        O.gepp_solve([[1.0, 2.0], [2.0, 4.0]], [1.0, 1.0])


# ---------------------------------------------------------- printed table

def _remez_cond(lo, u):
    a, b, c, info = O.optimal_quintic(lo, u, return_info=True)
    if info["shortcut"]:
        return None
    x1, x2 = info["x1"], info["x2"]
    M = np.array([[x, x ** 3, x ** 5, s] for x, s in ((lo, 1), (x1, -1), (x2, 1), (u, -1))])
    return np.linalg.cond(M)


def test_printed_table_l1e3():
    """App. A online listing: the 8 rows of coeffs_list (before safety).

    Rows from the Remez branch agree within 4 cond(M) eps (M = the final 4x4
    system, the backward-error bound of a pivoted solve). The printed row 8 is
    the unscaled Newton-Schulz quintic, while the solve returns it scaled to
    u_8 = 1 + O(1e-9): they agree within 5 (u_8 - 1)."""
    printed = read_golden("muon_table_l1e-3_d5.txt")
    rows, bounds, info = O.optimal_composition(1e-3, 8, return_info=True)
    raw = info["raw"]
    for t in range(8):
        lt, ut = bounds[t]
        lo = max(lt, O.KAPPA * ut)
        cond = _remez_cond(lo, ut)
        rel = max(abs(p - q) / abs(p) for p, q in zip(printed[t], raw[t]))
        if cond is None:
            assert info["shortcut"][t]
            assert rel <= 5 * (ut - 1.0) + 4 * EPS
        else:
            assert rel <= 4 * cond * EPS, (t, rel, cond)
    # rows 1..7 come from the Remez branch and row 8 from the shortcut, so the
    # default safety rule reproduces the listing's "all rows but the last"
    assert info["shortcut"] == [False] * 7 + [True]


def test_safety_matches_listing():
    raw_rows, _ = O.optimal_composition(1e-3, 8, safety=1.0)
    rows, _ = O.optimal_composition(1e-3, 8, safety=1.01)
    for t in range(7):
        a, b, c = raw_rows[t]
        assert rows[t] == (a / 1.01, b / (1.01 * 1.01 * 1.01), c / (1.01 * 1.01 * 1.01 * 1.01 * 1.01))
    assert rows[7] == raw_rows[7]
    rows_sl, _ = O.optimal_composition(1e-2, 4, safety=1.01, safety_skip_last=True)
    raw4, _ = O.optimal_composition(1e-2, 4)
    assert rows_sl[3] == raw4[3] and rows_sl[0] != raw4[0]


# ------------------------------------------------------ equioscillation

CASES = [(O.KAPPA, 1.0), (1e-7, 1.0), (1e-3, 1.0), (0.03, 1.0), (0.2, 1.3),
         (0.5, 1.0), (0.9, 1.0), (0.99, 1.0), (0.9999, 1.0), (2.0, 5.0)]


@pytest.mark.parametrize("l,u", CASES)
def test_equioscillation(l, u):
    """Lemma (App. D): the minimax odd quintic equioscillates at q+2 = 4
    points {l, x1, x2, u} with 1 - p = +E, -E, +E, -E, and |1 - p| <= |E| on
    [l, u]."""
    a, b, c, info = O.optimal_quintic(l, u, return_info=True)
    assert not info["shortcut"]
    E = info["E"]
    pts = [l, info["x1"], info["x2"], u]
    sgn = [1, -1, 1, -1]
    for x, s in zip(pts, sgn):
        assert abs((1 - p_eval((a, b, c), x)) - s * E) <= 1e-14 * max(1.0, abs(a) * u), (x, E)
    assert l < pts[1] < pts[2] < u
    # interior points are stationary
    for x in pts[1:3]:
        assert abs(dp_eval((a, b, c), x)) <= 1e-6 * abs(a)
    g = dense_grid(l, u)
    err = np.max(np.abs(1 - p_eval((a, b, c), g)))
    assert err <= abs(E) + 1e-13
    assert err >= abs(E) - 1e-13


def test_remez_iterations_at_most_five():
    """App. F: the degree-5 Remez loop never needed more than five iterations
    in the paper's experiments."""
    worst = 0
    for l in [1e-7, 1e-5, 1e-4, 1e-3, 1e-2, 0.03, 0.1, 0.3]:
        rows, bounds = O.optimal_composition(l, 12)
        for (lt, ut) in bounds[:-1]:
            lo = max(lt, O.KAPPA * ut)
            _, _, _, info = O.optimal_quintic(lo, ut, return_info=True)
            worst = max(worst, info["iters"])
    assert 1 <= worst <= 5


def test_remez_iteration_cap():
    with pytest.raises(O.NoConvergence):
        O.optimal_quintic(1e-3, 1.0, max_iters=1)


# ------------------------------------------------------------- LP pin

def _lp_minimax(l, u, degree, n=4001):
    from scipy.optimize import linprog
    # Chebyshev-clustered grid on [l, u]
    k = np.arange(n)
    x = 0.5 * (l + u) - 0.5 * (u - l) * np.cos(np.pi * k / (n - 1))
    pw = [1, 3, 5][: (degree + 1) // 2]
    V = np.stack([x ** p for p in pw], axis=1)
    nv = V.shape[1]
    # variables: coeffs..., t ; minimise t s.t. -t <= 1 - V c <= t
    cvec = np.zeros(nv + 1)
    cvec[-1] = 1.0
    A1 = np.hstack([-V, -np.ones((n, 1))])   # 1 - Vc <= t  ->  -Vc - t <= -1
    A2 = np.hstack([V, -np.ones((n, 1))])    # Vc - 1 <= t  ->   Vc - t <= 1
    A = np.vstack([A1, A2])
    bvec = np.concatenate([-np.ones(n), np.ones(n)])
    res = linprog(cvec, A_ub=A, b_ub=bvec, bounds=[(None, None)] * (nv + 1), method="highs")
    assert res.status == 0
    return res.x[:-1], res.x[-1]


@pytest.mark.parametrize("l,u", [(O.KAPPA, 1.0), (1e-3, 1.0), (0.1, 1.0), (0.5, 1.0), (0.3, 2.0)])
def test_quintic_matches_lp(l, u):
    pytest.importorskip("scipy")
    a, b, c, info = O.optimal_quintic(l, u, return_info=True)
    coef, t = _lp_minimax(l, u, 5)
    E = abs(info["E"])
    assert t <= E + 1e-12            # the grid is a subset of [l, u]
    assert t >= E - 1e-6 * max(E, 1e-3)   # grid discretisation
    assert np.allclose(coef, [a, b, c], rtol=1e-5, atol=1e-7 * abs(a))


@pytest.mark.parametrize("l,u", [(0.1, 1.0), (1e-3, 1.0), (0.5, 1.0), (0.25, 3.0)])
def test_cubic_matches_lp_and_equioscillates(l, u):
    pytest.importorskip("scipy")
    a, b = O.optimal_cubic(l, u)
    alpha = math.sqrt(3.0 / (u * u + l * u + l * l))
    beta = 4.0 / (2.0 + l * u * (l + u) * alpha ** 3)
    E = beta - 1.0
    p = lambda x: a * x + b * x ** 3
    # Eq. equioscillation_deg_3: p(l) = 1-E, p(1/alpha) = 1+E, p(u) = 1-E
    assert abs(p(l) - (1 - E)) <= 1e-14
    assert abs(p(1 / alpha) - (1 + E)) <= 1e-14
    assert abs(p(u) - (1 - E)) <= 1e-14
    assert abs(math.sqrt(-a / (3 * b)) - 1 / alpha) <= 1e-14
    coef, t = _lp_minimax(l, u, 3)
    assert abs(t - E) <= 1e-6 * max(E, 1e-3)
    assert np.allclose(coef, [a, b], rtol=1e-5)


def test_cubic_degenerate_interval_is_ns3():
    # l = u: alpha = 1/u, beta = 1, p = p_NS(x/u)
    a, b = O.optimal_cubic(2.0, 2.0)
    assert abs(a - 1.5 / 2.0) < 1e-15 and abs(b + 0.5 / 8.0) < 1e-15


# ----------------------------------------------------------- l/u -> 1

@pytest.mark.parametrize("gap", [1e-2, 1e-3, 1e-4])
def test_ns_limit(gap):
    """App. F: max |p* - p_NS(x/u)| <= 2 max |1 - p_NS(x/u)| on [l, u]
    (triangle inequality plus optimality of p*). The paper then bounds the
    right side by 2 (1 - l/u)^3; the exact NS5 error at x = 1 - d is
    d^3 (8 + 9x + 3x^2) / 8, so that last step holds only up to a constant
    (<= 5 (1 - l/u)^3), which is what is checked here."""
    u = 1.0
    l = u * (1 - gap)
    a, b, c = O.optimal_quintic(l, u)
    g = dense_grid(l, u, 20001)
    ns = (g / u) * (15 - 10 * (g / u) ** 2 + 3 * (g / u) ** 4) / 8
    diff = np.max(np.abs(p_eval((a, b, c), g) - ns))
    assert diff <= 2 * np.max(np.abs(1 - ns)) + 1e-13
    assert diff <= 5 * gap ** 3 + 1e-13


def test_shortcut_branch():
    a, b, c = O.optimal_quintic(1.0 - 1e-6, 1.0)
    assert (a, b, c) == (1.875, -1.25, 0.375)
    a, b, c = O.optimal_quintic(2.0 * (1 - 1e-6), 2.0)
    assert a == 1.875 / 2 and b == -1.25 / 8 and c == 0.375 / 32


def test_kappa_is_ratio_ten():
    """The code's cushion kappa makes the first-step error E = 9/11, i.e. the
    cushioned polynomial's range ratio (1+E)/(1-E) is exactly 10."""
    _, _, _, info = O.optimal_quintic(O.KAPPA, 1.0, return_info=True)
    assert abs(info["E"] - 9.0 / 11.0) <= 1e-14


# --------------------------------------------------------- Thm. 1 greedy

@pytest.mark.parametrize("l,T,degree", [(1e-3, 8, 5), (1e-4, 6, 5), (1e-7, 12, 5), (0.03, 3, 5),
                                        (1e-3, 10, 3), (0.1, 5, 3)])
def test_greedy_bounds(l, T, degree):
    """Eq. newbounds / Lemma computable error: on [l_t, u_t] the recentred
    p_t has its minimum l_{t+1} = p_t(l_t) at l_t and its maximum
    2 - l_{t+1}."""
    rows, bounds = O.optimal_composition(l, T, degree=degree)
    for t in range(T):
        lt, ut = bounds[t]
        g = np.unique(np.concatenate([np.geomspace(lt, ut, 100001), np.linspace(lt, ut, 100001)]))
        v = p_eval(rows[t], g)
        ln = bounds[t + 1][0]
        assert abs(p_eval(rows[t], lt) - ln) <= 4 * EPS
        assert v.min() >= ln - 1e-13
        assert v.max() <= 2 - ln + 1e-12
        assert v.max() >= 2 - ln - 1e-7 * (1 - ln) - 1e-13


@pytest.mark.parametrize("l,T", [(1e-3, 5), (1e-3, 8), (1e-4, 6), (1e-7, 12)])
def test_composition_image(l, T):
    """The composed polynomial maps [l, 1] into [l_{T+1}, 2 - l_{T+1}], with
    the minimum attained at x = l."""
    rows, bounds = O.optimal_composition(l, T)
    g = np.unique(np.concatenate([np.geomspace(l, 1.0, 200001), np.linspace(l, 1.0, 200001)]))
    v = O.compose_scalar(g, rows)
    lT = bounds[-1][0]
    # Near x = 1 each step's rounding is amplified by the later steps' slopes
    # at u_t (the instability the safety factor of Sec. 3.4 guards against),
    # so the upper tolerance is 8 eps sum_t prod_{s>=t} max(1, |p_s'(u_s)|).
    amp, tot = 1.0, 0.0
    for t in range(T - 1, -1, -1):
        amp *= max(1.0, abs(dp_eval(rows[t], bounds[t][1])))
        tot += amp
    assert v.min() >= lT - 1e-12
    assert v.max() <= 2 - lT + 8 * EPS * tot + 1e-12
    assert abs(O.compose_scalar(np.array([l]), rows)[0] - lT) <= 1e-12


def _max_err_composed(rows, l, u=1.0, n=100001):
    g = np.unique(np.concatenate([np.geomspace(l, u, n), np.linspace(l, u, n)]))
    return float(np.max(np.abs(1 - O.compose_scalar(g, rows))))


@pytest.mark.parametrize("l,T", [(1e-2, 1), (1e-2, 3), (1e-3, 4), (0.1, 2)])
def test_greedy_is_optimal_uncushioned(l, T):
    """Thm. 1: without cushioning the greedy composition is optimal, its
    error is 1 - l_{T+1}, it beats Newton-Schulz and Jordan, and perturbing
    any one coefficient makes it worse."""
    rows, bounds = O.optimal_composition(l, T, cushion=0.0)
    best = _max_err_composed(rows, l)
    assert abs(best - (1 - bounds[-1][0])) <= 1e-9
    assert best <= _max_err_composed(O.newton_schulz5_table(T), l) + 1e-12
    # Jordan's polynomial is unnormalised; scale-optimise it for fairness
    assert best <= _max_err_composed(O.jordan_table(T), l) + 1e-12
    rng = np.random.default_rng(1)
    for _ in range(40):
        t = rng.integers(T)
        j = rng.integers(3)
        pert = [list(r) for r in rows]
        pert[t][j] *= 1 + rng.choice([-1, 1]) * 10 ** rng.uniform(-6, -3)
        assert _max_err_composed(pert, l) >= best - 1e-10


def test_cushioned_still_beats_ns5():
    for l, T in [(1e-3, 5), (1e-4, 6), (1e-7, 12)]:
        rows, bounds = O.optimal_composition(l, T)
        assert 1 - bounds[-1][0] < _max_err_composed(O.newton_schulz5_table(T), l)


@pytest.mark.parametrize("l,T,degree", [(0.1, 1, 5), (0.1, 2, 5), (0.05, 3, 5), (0.3, 2, 3), (0.1, 3, 3)])
def test_thm2_bound(l, T, degree):
    """Thm. 2: ||polar(M) - X_T||_2 <= (1 - l^2)^((q+1)^T), d = 2q+1."""
    q = (degree - 1) // 2
    rows, bounds = O.optimal_composition(l, T, degree=degree, cushion=0.0)
    assert 1 - bounds[-1][0] <= (1 - l * l) ** ((q + 1) ** T) + 1e-15


# ------------------------------------------------------- App. G facts

def test_safety_fixed_point():
    """App. G: with p -> p(x/1.01) the NS quintic's fixed point is 0.999998."""
    x = 1.0
    for _ in range(200):
        y = x / 1.01
        x = (15 * y - 10 * y ** 3 + 3 * y ** 5) / 8
    assert abs(x - 0.999998) <= 5e-7


def test_fig7_unstabilised_polynomial():
    """Fig. 7: the optimal quintic on [0.005, 1] sends values near 0.8 almost
    to zero and has slope about 25 at u = 1 (1 + eps -> u_{t+1} + 25 eps)."""
    a, b, c, info = O.optimal_quintic(0.005, 1.0, return_info=True)
    x2 = info["x2"]
    assert 0.7 < x2 < 0.9
    assert p_eval((a, b, c), x2) < 0.1
    slope = dp_eval((a, b, c), 1.0)
    assert 20 < slope < 30


@pytest.mark.parametrize("l,T", [(1e-3, 8), (1e-4, 6), (0.005, 3)])
def test_safety_keeps_overshoot_bounded(l, T):
    """Fig. 7 caption: with the safety factor every x <= 1.01 u_t is mapped
    to at most u_{t+1} (checked on the rows that carry the factor)."""
    rows, bounds, info = O.optimal_composition(l, T, safety=1.01, return_info=True)
    for t in range(T):
        if info["shortcut"][t]:
            continue
        lt, ut = bounds[t]
        g = np.linspace(0.0, 1.01 * ut, 200001)
        assert p_eval(rows[t], g).max() <= bounds[t + 1][1] + 1e-12


def test_fig9_five_step_map():
    """Fig. 9 bottom panel: the paper's five-step table (with safety) maps
    singular values >= 1e-3 close to 1 and values <= 1e-4 close to 0."""
    printed = read_golden("muon_table_l1e-3_d5.txt")
    tab = [(a / 1.01, b / 1.01 ** 3, c / 1.01 ** 5) for (a, b, c) in printed[:5]]
    hi = O.compose_scalar(np.geomspace(1e-3, 1.0, 20001), tab)
    lo = O.compose_scalar(np.geomspace(1e-7, 1e-4, 2001), tab)
    assert hi.min() >= 0.8 and hi.max() <= 1.2
    assert lo.max() <= 0.15


def test_argument_errors():
    with pytest.raises(ValueError):
        O.optimal_composition(0.0, 5)
    with pytest.raises(ValueError):
        O.optimal_composition(1e-3, 0)
    with pytest.raises(ValueError):
        O.optimal_composition(1e-3, 5, degree=7)
    with pytest.raises(ValueError):
        O.optimal_composition(1e-3, 5, safety=0.5)
