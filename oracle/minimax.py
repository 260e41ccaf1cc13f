"""Offline stage of Polar Express in plain FP64 Python floats (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's offline stage (Alg. 1, offline box; App. A offline code; App. F)
builds, for a lower bound l and T steps, the odd polynomials
p_t(x) = a_t x + b_t x^3 + c_t x^5 greedily (Thm. 1, Eq. greedy):

* l_1 = l, u_1 = 1;
* p_t is the minimax odd polynomial for the constant 1 on the cushioned
  interval [max(l_t, kappa u_t), u_t] (Sec. 3.4 and App. G, second fix);
* p_t is rescaled so that it is centred around 1 on [l_t, u_t], i.e. by
  2 / (p_t(l_t) + max p_t) (App. A offline code, recentring; for the quintic
  the maximum is p_t(u_t), for the cubic it is the interior extremum);
* l_{t+1} = p_t(l_t), u_{t+1} = 2 - l_{t+1} (Eq. newbounds);
* afterwards every row except those that came from the l/u -> 1 shortcut is
  replaced by p_t(x / safety) (Sec. 3.4 and App. G, first fix).

The degree-5 minimax polynomial comes from the simplified Remez iteration of
Alg. 3 (App. F): trial points {l, x1, x2, u}, a 4x4 linear solve for
(a, b, c, E) with alternating signs, new interior points from the quadratic
formula on 5c y^2 + 3b y + a = 0 (y = x^2), stop once E stops changing. The
degree-3 one is the closed form of Eq. deg3_solution.

Arithmetic contract (so that an independent implementation in another
language can reproduce these values bit for bit):

* powers are repeated products evaluated left to right:
  x3 = (x*x)*x, x5 = (((x*x)*x)*x)*x;
* a polynomial value is ((a*x) + (b*x3)) + (c*x5);
* the 4x4 system is solved by Gaussian elimination with partial pivoting
  (first row of largest |pivot|), eliminating rows below the pivot in natural
  order, then back substitution from the last row;
* sqrt is the correctly rounded IEEE square root; no fused multiply-add.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

#: Cushion factor used by the paper's offline code (App. A). With it the first
#: step's equioscillation error is 9/11, i.e. (1 + E) / (1 - E) = 10.
KAPPA = 0.02407327424182761
#: Alg. 1 cushions at u/10; used here for degree 3, where the code gives none.
KAPPA_DEG3 = 0.1
#: l/u threshold above which the minimax quintic equals the scaled
#: Newton-Schulz quintic to double precision (App. F; the code's constant).
NS_SHORTCUT = 1.0 - 5e-6
#: Remez stopping tolerance on |E_k - E_{k-1}| (the code's constant).
REMEZ_TOL = 1e-15
#: Iteration cap (the paper reports at most 5 iterations; App. F).
REMEZ_MAX_ITERS = 100


class NoConvergence(RuntimeError):
    pass


def _pow3(x: float) -> float:
    return x * x * x


def _pow5(x: float) -> float:
    return x * x * x * x * x


def eval_odd(a: float, b: float, c: float, x: float) -> float:
    """p(x) = a x + b x^3 + c x^5 in the contract's evaluation order."""
    return a * x + b * _pow3(x) + c * _pow5(x)


def gepp_solve(M: Sequence[Sequence[float]], y: Sequence[float]) -> List[float]:
    """Solve M z = y by Gaussian elimination with partial pivoting.

    This is the textbook algorithm written out, standing in for the
    ``np.linalg.solve`` call of the paper's offline code so that the result
    has a fixed rounding order.
    """
    n = len(M)
    A = [[float(v) for v in M[i]] + [float(y[i])] for i in range(n)]
    for k in range(n):
        p = k
        best = abs(A[k][k])
        for i in range(k + 1, n):
            if abs(A[i][k]) > best:
                best = abs(A[i][k])
                p = i
        if best == 0.0:
            raise ZeroDivisionError("singular system")
        if p != k:
            A[k], A[p] = A[p], A[k]
        piv = A[k][k]
        for i in range(k + 1, n):
            f = A[i][k] / piv
            for j in range(k + 1, n + 1):
                A[i][j] = A[i][j] - f * A[k][j]
    z = [0.0] * n
    for i in range(n - 1, -1, -1):
        acc = A[i][n]
        for j in range(i + 1, n):
            acc = acc - A[i][j] * z[j]
        z[i] = acc / A[i][i]
    return z


def optimal_quintic(l: float, u: float, max_iters: int = REMEZ_MAX_ITERS,
                    return_info: bool = False):
    """Minimax odd quintic for x -> 1 on [l, u] (Alg. 3, App. F).

    Returns (a, b, c) or, with ``return_info``, (a, b, c, info) where info
    holds the final trial points, the signed error E, the iteration count and
    whether the l/u -> 1 shortcut was taken.
    """
    if not (l > 0.0 and u > 0.0):
        raise ValueError("need 0 < l, 0 < u")
    # Once the greedy bounds have converged in FP64, rounding can leave
    # l_t slightly above u_t = 2 - l_t; that interval is treated as
    # degenerate and takes the shortcut like any l/u >= NS_SHORTCUT.
    if l / u >= NS_SHORTCUT:
        # Scaled Newton-Schulz quintic (x/u)(15 - 10(x/u)^2 + 3(x/u)^4)/8.
        a, b, c = (15.0 / 8.0) / u, (-10.0 / 8.0) / _pow3(u), (3.0 / 8.0) / _pow5(u)
        info = dict(shortcut=True, iters=0, E=None, x1=None, x2=None)
        return (a, b, c, info) if return_info else (a, b, c)
    x1 = (3.0 * l + u) / 4.0
    x2 = (l + 3.0 * u) / 4.0
    E = math.inf
    E_old = None
    it = 0
    a = b = c = 0.0
    pts = (x1, x2)
    while E_old is None or abs(E_old - E) > REMEZ_TOL:
        if it >= max_iters:
            raise NoConvergence(f"Remez did not converge on [{l}, {u}]")
        E_old = E
        pts = (x1, x2)
        rows = [
            [l, _pow3(l), _pow5(l), 1.0],
            [x1, _pow3(x1), _pow5(x1), -1.0],
            [x2, _pow3(x2), _pow5(x2), 1.0],
            [u, _pow3(u), _pow5(u), -1.0],
        ]
        a, b, c, E = gepp_solve(rows, [1.0, 1.0, 1.0, 1.0])
        disc = 9.0 * (b * b) - 20.0 * a * c
        sq = math.sqrt(disc)
        x1 = math.sqrt((-3.0 * b - sq) / (10.0 * c))
        x2 = math.sqrt((-3.0 * b + sq) / (10.0 * c))
        it += 1
    info = dict(shortcut=False, iters=it, E=E, x1=pts[0], x2=pts[1])
    return (a, b, c, info) if return_info else (a, b, c)


def optimal_cubic(l: float, u: float) -> Tuple[float, float]:
    """Minimax odd cubic for x -> 1 on [l, u], Eq. deg3_solution:
    p(x) = beta * p_NS(alpha x), p_NS(x) = 3/2 x - 1/2 x^3,
    alpha = sqrt(3 / (u^2 + l u + l^2)), beta = 4 / (2 + l u (l + u) alpha^3)."""
    if not (l > 0.0 and u > 0.0):
        raise ValueError("need 0 < l, 0 < u")
    alpha = math.sqrt(3.0 / (u * u + l * u + l * l))
    alpha3 = _pow3(alpha)
    beta = 4.0 / (2.0 + l * u * (l + u) * alpha3)
    return 1.5 * beta * alpha, -0.5 * beta * alpha3


def _cubic_beta(l: float, u: float) -> float:
    alpha = math.sqrt(3.0 / (u * u + l * u + l * l))
    return 4.0 / (2.0 + l * u * (l + u) * _pow3(alpha))


def optimal_composition(l: float, T: int, degree: int = 5, cushion: float | None = None,
                        safety: float = 1.0, safety_skip_last: bool = False,
                        return_info: bool = False):
    """Greedy composition of Thm. 1 with the paper's stabilisations.

    Returns ``rows`` (T tuples (a, b, c); c = 0 for degree 3) and ``bounds``
    (T+1 pairs (l_t, u_t), from the recentred rows before the safety factor).

    Safety reading: row t is replaced by p_t(x / safety) unless its unscaled
    polynomial came from the l/u -> 1 shortcut (for degree 3: unless the
    cushioned interval has l/u >= NS_SHORTCUT). With ``safety_skip_last`` the
    last row is left unscaled as well (App. G: may be omitted in the final
    iteration).
    """
    if degree not in (3, 5):
        raise ValueError("degree must be 3 or 5")
    if T < 1:
        raise ValueError("T >= 1")
    if not (0.0 < l <= 1.0):
        raise ValueError("need 0 < l <= 1")
    if safety < 1.0:
        raise ValueError("safety >= 1")
    if cushion is None:
        cushion = KAPPA if degree == 5 else KAPPA_DEG3
    u = 1.0
    raw = []
    shortcut = []
    bounds = [(l, u)]
    for _ in range(T):
        lo = max(l, cushion * u)
        if degree == 5:
            a, b, c, info = optimal_quintic(lo, u, return_info=True)
            sc = info["shortcut"]
        else:
            a, b = optimal_cubic(lo, u)
            c = 0.0
            sc = lo / u >= NS_SHORTCUT
        pl = eval_odd(a, b, c, l)
        if degree == 5:
            # the quintic's equioscillation ends on a maximum at u
            pmax = eval_odd(a, b, c, u)
        else:
            # the cubic's ends on a minimum at u; its maximum is the interior
            # extremum 1/alpha, where p = beta * p_NS(1) = beta
            pmax = _cubic_beta(lo, u)
        r = 2.0 / (pl + pmax)
        a = a * r
        b = b * r
        c = c * r
        raw.append((a, b, c))
        shortcut.append(sc)
        l = eval_odd(a, b, c, l)
        u = 2.0 - l
        bounds.append((l, u))
    s3 = safety * safety * safety
    s5 = s3 * safety * safety
    rows = []
    for t, (a, b, c) in enumerate(raw):
        skip = shortcut[t] or safety == 1.0 or (safety_skip_last and t == T - 1)
        if skip:
            rows.append((a, b, c))
        else:
            rows.append((a / safety, b / s3, c / s5))
    if return_info:
        return rows, bounds, dict(raw=raw, shortcut=shortcut)
    return rows, bounds


def newton_schulz5_table(T: int) -> List[Tuple[float, float, float]]:
    """Degree-5 Newton-Schulz, p(x) = (15x - 10x^3 + 3x^5)/8 (Sec. 1.2)."""
    return [(15.0 / 8.0, -10.0 / 8.0, 3.0 / 8.0)] * T


def jordan_table(T: int) -> List[Tuple[float, float, float]]:
    """Jordan's fixed quintic 3.4445x - 4.7750x^3 + 2.0315x^5 (Sec. 1.2)."""
    return [(3.4445, -4.7750, 2.0315)] * T
