"""Online stage of Polar Express in FP64, plus truth and error metrics (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``normalise``: X_0 = G / (1.01 ||G||_F + 1e-7), transposed when G has more
  rows than columns so that X_0 is s x L with s = min(m, n) (App. A online
  code; the Alg. 1 variant divides by ||G||_F + 1e-2 and is available through
  the ``scale`` / ``eps`` arguments).
* ``polar_express``: for each row (a, b, c): A = X X^T, B = b A + c A A,
  X = a X + B X (Sec. 3.5 Horner form, App. A online code), then transpose
  back. Plain numpy matmul in FP64; no blocking or fusion.
* ``polar_express_spectral``: the same map written through the SVD,
  U p(x) V^T with x the normalised singular values (Sec. 2 definition of p(M)
  and App. C), for inputs whose factors are known.
* ``fast_rectangular``: Alg. 4 (the appendix on fast polynomial iteration for
  rectangular matrices): Y = X X^T, Q_t = Q_{t-1} h_t(Q^T Y Q), X_T = Q_T X,
  restarted every few steps, with the shift Y + 1e-3 I in the first block;
  ``fast_rectangular_spectral`` is the same map on the singular values.
* ``polar_svd``: polar(G) = U V^T (Eq. matrixsign).
* error metrics: ||X - polar(G)||_F / sqrt(min(m, n)), max_i |sigma_i(X) - 1|,
  their restriction to singular directions with sigma_i(G) >= gamma sigma_max
  (App. H.1, convergence of the top singular values), and the relative
  Frobenius distance used for GPU-vs-oracle parity.
"""
from __future__ import annotations

import math
from typing import Iterable, Sequence, Tuple

import numpy as np

NORM_SCALE = 1.01
NORM_EPS = 1e-7


def normalise(G: np.ndarray, scale: float = NORM_SCALE, eps: float = NORM_EPS):
    """Return (X0, transposed): X0 is s x L (s = min(m, n))."""
    G = np.asarray(G, dtype=np.float64)
    nu = math.sqrt(float(np.sum(G * G)))
    X = G / (scale * nu + eps)
    transposed = G.shape[0] > G.shape[1]
    if transposed:
        X = X.T
    return np.ascontiguousarray(X), transposed


def polar_express(G: np.ndarray, table: Iterable[Sequence[float]],
                  scale: float = NORM_SCALE, eps: float = NORM_EPS,
                  return_steps: bool = False):
    """FP64 Polar Express iteration; returns an m x n array like G."""
    X, transposed = normalise(G, scale, eps)
    steps = []
    for (a, b, c) in table:
        A = X @ X.T
        B = b * A + c * (A @ A)
        X = a * X + B @ X
        if return_steps:
            steps.append(X.T.copy() if transposed else X.copy())
    out = X.T if transposed else X
    out = np.ascontiguousarray(out)
    return (out, steps) if return_steps else out


FAST_SHIFT = 1e-3      # stabiliser of the first application (appendix on rectangular matrices)
FAST_EPS = 1e-3        # normalisation offset used with it


def fast_rectangular(G: np.ndarray, table: Iterable[Sequence[float]], restart: int = 3,
                     shift: float = FAST_SHIFT, scale: float = NORM_SCALE, eps: float = FAST_EPS,
                     return_blocks: bool = False):
    """Alg. 4 (fast polynomial iteration for rectangular matrices) in FP64, on
    the short side: X s x L, p_t(X) = h_t(X X^T) X with h_t(y) = a + b y + c y^2.

    The steps are taken in blocks of ``restart`` (the restarting strategy of
    the same appendix; restart = 1 is the baseline iteration). For a block:
    Y = X X^T (+ shift I in the first block only), Q = I, then per step
    R = Q^T Y Q and Q = Q h(R); finally X = Q X. The normalisation divides by
    scale ||G||_F + eps (the appendix uses ||X||_F + 1e-3 with the shift)."""
    X, transposed = normalise(G, scale, eps)
    s = X.shape[0]
    rows = [tuple(r) for r in table]
    blocks = []
    t = 0
    first = True
    while t < len(rows):
        Y = X @ X.T
        if first and shift:
            Y = Y + shift * np.eye(s)
        Q = np.eye(s)
        for (a, b, c) in rows[t:t + restart]:
            R = Q.T @ Y @ Q
            H = a * np.eye(s) + b * R + c * (R @ R)
            Q = Q @ H
        X = Q @ X
        t += restart
        first = False
        if return_blocks:
            blocks.append(X.T.copy() if transposed else X.copy())
    out = np.ascontiguousarray(X.T if transposed else X)
    return (out, blocks) if return_blocks else out


def fast_rectangular_spectral(U: np.ndarray, s: np.ndarray, V: np.ndarray, table, restart: int = 3,
                              shift: float = FAST_SHIFT, scale: float = NORM_SCALE, eps: float = FAST_EPS):
    """The map of ``fast_rectangular`` on G = U diag(s) V^T written through the
    singular values: with x = s / (scale ||s|| + eps), every block takes
    y = x^2 (+ shift in the first block), q = 1, and per step
    q <- q h(y q^2); then x <- x q. (Y, Q, R are polynomials of one symmetric
    matrix, so the recursion acts on each eigenvalue separately.)"""
    x = np.asarray(s, dtype=np.float64) / (scale * math.sqrt(float(np.sum(np.asarray(s, np.float64) ** 2))) + eps)
    rows = [tuple(r) for r in table]
    t = 0
    first = True
    while t < len(rows):
        y = x * x + (shift if first and shift else 0.0)
        q = np.ones_like(x)
        for (a, b, c) in rows[t:t + restart]:
            r = y * q * q
            q = q * (a + b * r + c * r * r)
        x = x * q
        t += restart
        first = False
    return (U * x) @ V.T


def compose_scalar(x, table: Iterable[Sequence[float]]):
    """Scalar composition p_T(...p_1(x)) for an array of x."""
    x = np.asarray(x, dtype=np.float64)
    for (a, b, c) in table:
        y = x * x
        x = x * (a + y * (b + c * y))
    return x


def polar_express_spectral(U: np.ndarray, s: np.ndarray, V: np.ndarray,
                           table: Iterable[Sequence[float]],
                           scale: float = NORM_SCALE, eps: float = NORM_EPS,
                           rows: np.ndarray | None = None, cols: np.ndarray | None = None):
    """U diag(p(x)) V^T with x = s / (scale ||s||_2 + eps).

    With ``rows``/``cols`` index arrays, returns only those sampled entries
    (each costs O(k)), which serves parity at sizes where the dense FP64
    iteration is too slow.
    """
    s = np.asarray(s, dtype=np.float64)
    nu = math.sqrt(float(np.sum(s * s)))
    px = compose_scalar(s / (scale * nu + eps), table)
    if rows is None:
        return (U * px[None, :]) @ V.T
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    return np.einsum("ik,k,ik->i", U[rows], px, V[cols])


def polar_svd(G: np.ndarray) -> np.ndarray:
    """polar(G) = U V^T from the reduced SVD (LAPACK)."""
    U, _, Vt = np.linalg.svd(np.asarray(G, dtype=np.float64), full_matrices=False)
    return U @ Vt


def polar_2x2(M: np.ndarray) -> np.ndarray:
    """Closed-form polar factor of a nonsingular real 2x2 matrix:
    (M + sgn(det M) cof(M)) / sqrt(||M||_F^2 + 2 |det M|), cof = [[d,-c],[-b,a]]."""
    (a, b), (c, d) = np.asarray(M, dtype=np.float64)
    det = a * d - b * c
    sg = 1.0 if det > 0 else -1.0
    cof = np.array([[d, -c], [-b, a]])
    return (np.asarray(M, dtype=np.float64) + sg * cof) / math.sqrt(a * a + b * b + c * c + d * d + 2 * abs(det))


def err_polar_fro(X: np.ndarray, P: np.ndarray) -> float:
    """||X - P||_F / sqrt(min(m, n)) (so that ||P||_F / sqrt(min) = 1)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(X - P) / math.sqrt(min(X.shape)))


def max_sigma_err(X: np.ndarray) -> float:
    """max_i |sigma_i(X) - 1| over the min(m, n) singular values."""
    sv = np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)
    return float(np.max(np.abs(sv - 1.0)))


def restricted_errors(X: np.ndarray, U: np.ndarray, s: np.ndarray, V: np.ndarray,
                      gamma: float = 1e-3) -> Tuple[float, float]:
    """Errors restricted to the singular directions of G with
    s_i >= gamma * max(s): compares U1 U1^T X V1 V1^T with U1 V1^T.

    Returns (||U1^T X V1 - I||_F / sqrt(k1), max_i |sigma_i(U1^T X V1) - 1|).
    """
    s = np.asarray(s)
    keep = s >= gamma * np.max(s)
    U1 = U[:, keep]
    V1 = V[:, keep]
    C = U1.T @ np.asarray(X, dtype=np.float64) @ V1
    k1 = C.shape[0]
    fro = float(np.linalg.norm(C - np.eye(k1)) / math.sqrt(k1))
    sv = np.linalg.svd(C, compute_uv=False)
    return fro, float(np.max(np.abs(sv - 1.0)))


def rel_fro(X: np.ndarray, Y: np.ndarray) -> float:
    """||X - Y||_F / ||Y||_F."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))
