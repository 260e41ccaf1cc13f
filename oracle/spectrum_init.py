"""Spectrum-aware initialisation for matrices with a large top singular value
(App. H, the case k = 1), in FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``power_bound``: a lower bound z <= sigma_1(X) from subspace iteration with
  one vector (the power method) on X^T X, started from a given vector v0:
  v <- X^T X v / ||X^T X v|| repeated ``iters`` times, then z = ||X v||. For
  any unit v, ||X v||^2 = v^T X^T X v <= sigma_1^2 (Rayleigh quotient; the
  paper's Cauchy-interlacing argument for k = 1). The random start is an input
  of the method, so both implementations take it from the caller.
* ``init_cubic``: with f = ||X||_F, the Frobenius identity of App. H gives
  sigma_1 in [z, f] and sigma_2, ..., sigma_n <= w = sqrt(f^2 - z^2). When the
  two intervals are disjoint (z > w), the odd cubic p(x) = a x + b x^3 with
  p(w) = p(z) = 1 is the paper's Eq. init_poly, written there for f = 1; for
  another f it is the same polynomial of x / f (Eq. init_poly at z / f, then
  a / f and b / f^3).
* ``spectrum_aware_table``: when the cubic applies, it is the first row
  (a, b, 0), followed by the Polar Express composition for the interval the
  cubic leaves, [l', 1] with l' = min(l / w, p(f)): p lies above the chord
  x / w on [0, w] (concave and increasing there), so the tail's lower bound l
  becomes l / w, and p is decreasing on [z, f], so sigma_1 ends in [p(f), 1].
  Otherwise the table is the plain composition with T + 1 rows (the cubic
  counts as an iteration, as in the appendix's comparison).
* ``spectrum_aware_polar``: normalise (the online code's 1.01 ||G||_F + 1e-7),
  bound, table, then the ordinary iteration over that table (which treats the
  cubic row like any other: A = X X^T, B = b A, X = a X + B X).

Readings (the appendix leaves these open): the power method runs on the
normalised X_0; the cubic applies exactly when the appendix builds it, i.e.
when the intervals [0, w] and [z, f] are disjoint, read strictly (2 z^2 > f^2:
at equality Eq. init_poly divides by zero) and with w > 0 (z < f; at z = f it
is singular too). Two options are not the paper's and are off by default:
``z_safety`` shrinks z by a relative amount before use (a caller that
evaluates the bound in FP32 can keep it below sigma_1 despite rounding), and
``gate`` keeps the cubic only when the greedy lower bound its composition
reaches after the last step beats that of the plain composition with one
more step.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from .iteration import NORM_EPS, NORM_SCALE, normalise, polar_express
from .minimax import optimal_composition

Z_SAFETY = 0.0   # the paper uses z as computed


def power_bound(X: np.ndarray, v0: Sequence[float], iters: int) -> float:
    """z = ||X v|| after ``iters`` normalised power steps v <- X^T X v from v0
    (v0 has X.shape[1] entries); z <= sigma_1(X) for every iters >= 0."""
    X = np.asarray(X, dtype=np.float64)
    v = np.asarray(v0, dtype=np.float64).copy()
    nv = float(np.linalg.norm(v))
    if nv == 0.0:
        raise ValueError("v0 must be nonzero")
    v /= nv
    for _ in range(iters):
        w = X.T @ (X @ v)
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(np.linalg.norm(X @ v))


def init_cubic_unit(z: float) -> Tuple[float, float]:
    """(a, b) of Eq. init_poly for ||M||_F = 1 and the bound z in (1/sqrt 2, 1)."""
    w = math.sqrt(1.0 - z * z)
    den = z * w * (2.0 * z * z - 1.0)
    a = (z * z * (z + w) - w) / den
    b = (w - z) / den
    return a, b


def init_cubic(z: float, f: float) -> Optional[Tuple[float, float, float]]:
    """(a, b, w) of the cubic through (w, 1) and (z, 1), w = sqrt(f^2 - z^2),
    or None when the intervals [0, w] and [z, f] are not disjoint."""
    if not (f > 0.0 and z > 0.0) or 2.0 * z * z <= f * f:
        return None
    zn = min(z / f, 1.0)
    if zn >= 1.0:
        return None                          # w = 0: Eq. init_poly is singular
    a1, b1 = init_cubic_unit(zn)
    return a1 / f, b1 / f ** 3, f * math.sqrt(1.0 - zn * zn)


def spectrum_aware_table(z: float, f: float, l: float, T: int, safety: float = 1.01,
                         z_safety: float = Z_SAFETY, gate: bool = False):
    """(table, info): the cubic row plus T Polar Express rows for [l', 1]
    when the cubic applies (App. H), else the plain composition with T + 1
    rows. With ``gate`` the cubic is kept only if the lower bound it leaves
    after its T steps, l'_T, exceeds the plain composition's l_{T+1} (the
    greedy bounds of Thm. 1)."""
    zs = z * (1.0 - z_safety)
    cub = init_cubic(zs, f)
    plain, pbounds = optimal_composition(l, T + 1, safety=safety)
    info = {"applied": False, "z": zs, "f": f, "l_after": l, "l_final_plain": pbounds[-1][0]}
    if cub is not None:
        a, b, w = cub
        pf = f * (a + b * f * f)
        lp = min(l / w, pf)
        if T > 0:
            rest, rbounds = optimal_composition(lp, T, safety=safety)
            l_final = rbounds[-1][0]
        else:
            rest, l_final = [], lp
        info.update({"w": w, "a": a, "b": b, "p_f": pf, "l_final_init": l_final})
        if not gate or l_final > pbounds[-1][0]:
            table: List[Tuple[float, float, float]] = [(a, b, 0.0)] + [tuple(r) for r in rest]
            info.update({"applied": True, "l_after": lp})
            return table, info
    return [tuple(r) for r in plain], info


def spectrum_aware_polar(G: np.ndarray, l: float, T: int, v0: Sequence[float], iters: int,
                         safety: float = 1.01, z_safety: float = Z_SAFETY, gate: bool = False):
    """App. H initialisation followed by T Polar Express steps; returns
    (X, table, info). X_0 is the s x L normalised matrix (short side first);
    the power method runs on the s x s matrix X_0 X_0^T, so v0 has
    s = min(m, n) entries and z = ||X_0^T v||."""
    X0, _ = normalise(G, NORM_SCALE, NORM_EPS)
    f = float(np.linalg.norm(X0))
    z = power_bound(X0.T, v0, iters)
    table, info = spectrum_aware_table(z, f, l, T, safety, z_safety, gate)
    return polar_express(G, table), table, info
