"""Seeded synthetic inputs for the polar-factor workloads.

This module is shared by the tests, ``bench.py`` and the smoke check. It holds
no arithmetic of the polar-factor method itself: it only draws matrices with a
prescribed singular structure (Haar-random singular vectors, chosen spectra,
Gaussian entries, low-rank spikes), in FP64 on the CPU, from
``numpy.random.default_rng(seed)``.

The workloads stand in for the gradient matrices of the paper's experiments
(Sec. 4.1 synthetic convergence study; Sec. 4.2 GPT-2 Muon runs), which are not
available here. Each generator states the shapes and distributions it draws.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------
# primitive draws
# --------------------------------------------------------------------------

def haar_orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """A rows x cols matrix with orthonormal columns (rows >= cols), Haar
    distributed on the Stiefel manifold: reduced QR of a Gaussian matrix with
    the column signs fixed by the sign of diag(R)."""
    if cols > rows:
        raise ValueError("haar_orthonormal needs rows >= cols")
    z = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(z, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def spectrum_gpt2(rng: np.random.Generator, k: int) -> np.ndarray:
    """s_i = 1/i + 1e-3 |N(0,1)|, i = 1..k (a decaying, gradient-like spectrum)."""
    i = np.arange(1, k + 1, dtype=np.float64)
    return 1.0 / i + 1e-3 * np.abs(rng.standard_normal(k))


def spectrum_loguniform(rng: np.random.Generator, k: int, lo: float, hi: float) -> np.ndarray:
    """k i.i.d. values, uniform in log10 on [lo, hi], sorted descending."""
    e = rng.uniform(np.log10(lo), np.log10(hi), size=k)
    return np.sort(10.0 ** e)[::-1].copy()


def spectrum_logspaced(k: int, lo: float, hi: float) -> np.ndarray:
    """k values evenly spaced in log10 from hi down to lo (Sec. 4.1 study)."""
    return np.logspace(np.log10(hi), np.log10(lo), k)


@dataclasses.dataclass
class SVDMatrix:
    """G = U diag(s) V^T with U (m x k), V (n x k) orthonormal, k = min(m, n)."""
    G: np.ndarray
    U: np.ndarray
    s: np.ndarray
    V: np.ndarray


def svd_matrix(rng: np.random.Generator, m: int, n: int, s: np.ndarray) -> SVDMatrix:
    k = min(m, n)
    s = np.asarray(s, dtype=np.float64)
    if s.shape != (k,):
        raise ValueError("spectrum length must be min(m, n)")
    U = haar_orthonormal(rng, m, k)
    V = haar_orthonormal(rng, n, k)
    G = (U * s[None, :]) @ V.T
    return SVDMatrix(G=G, U=U, s=s, V=V)


def gaussian(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    return rng.standard_normal((m, n))


def gaussian_plus_spike(rng: np.random.Generator, m: int, n: int, rank: int = 8,
                        spike_norm: float = 10.0) -> np.ndarray:
    """Z + P: Z has i.i.d. N(0,1) entries, P = c * Uk Vk^T with Haar Uk, Vk of
    rank ``rank`` and ||P||_F = spike_norm * ||Z||_F (the spike norm is taken
    relative to the noise so that the spike stands above the noise bulk at
    every size)."""
    z = rng.standard_normal((m, n))
    r = min(rank, m, n)
    uk = haar_orthonormal(rng, m, r)
    vk = haar_orthonormal(rng, n, r)
    p = uk @ vk.T  # ||p||_F = sqrt(r)
    p *= spike_norm * np.linalg.norm(z) / np.sqrt(r)
    return z + p


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    matrices: List[np.ndarray]             # FP64 inputs G_i (m_i x n_i)
    svd: List[Optional[SVDMatrix]]         # known factors where drawn that way
    l: float                               # lower bound used for the coefficients
    T: int                                 # polynomial steps
    dtype: str                             # "fp32" | "bf16" | "bf16x3"
    note: str = ""

    @property
    def shapes(self) -> List[Tuple[int, int]]:
        return [tuple(g.shape) for g in self.matrices]


def gpt2_small_shapes(layers: int = 12, d: int = 768) -> List[Tuple[int, int]]:
    """Per layer: attention qkv (d x 3d), attention proj (d x d), MLP fc
    (d x 4d) and MLP proj (4d x d)."""
    out = []
    for _ in range(layers):
        out += [(d, 3 * d), (d, d), (d, 4 * d), (4 * d, d)]
    return out


def d1024_shapes(layers: int = 24, d: int = 1024) -> List[Tuple[int, int]]:
    out = []
    for _ in range(layers):
        out += [(d, 3 * d), (d, d), (d, 4 * d), (4 * d, d)]
    return out


def plain_small(seed: int = 0) -> Workload:
    """One 256 x 128 matrix with i.i.d. N(0,1) entries, l = 1e-3, T = 8."""
    rng = np.random.default_rng(seed)
    g = gaussian(rng, 256, 128)
    return Workload("plain_256x128", [g], [None], 1e-3, 8, "fp32",
                    "256x128 iid N(0,1), seed 0")


def gpt2_small(layers: int = 12, d: int = 768, first_seed: int = 1) -> Workload:
    """The 48 hidden matrices of a 12-layer d=768 model. Each is
    U diag(s) V^T with Haar U, V, s_i = 1/i + 1e-3|N(0,1)|, scaled to unit
    Frobenius norm. Matrix j (0-based) uses seed first_seed + j."""
    mats, svds = [], []
    for j, (m, n) in enumerate(gpt2_small_shapes(layers, d)):
        rng = np.random.default_rng(first_seed + j)
        s = spectrum_gpt2(rng, min(m, n))
        s = s / np.linalg.norm(s)
        sv = svd_matrix(rng, m, n, s)
        mats.append(sv.G)
        svds.append(sv)
    return Workload("gpt2_small_muon_step", mats, svds, 1e-3, 5, "bf16",
                    f"{layers} layers x (d x 3d, d x d, d x 4d, 4d x d), d={d}")


def gpt2_heads_shapes(layers: int = 12, d: int = 768, heads: int = 12) -> List[Tuple[int, int]]:
    """Per-head splitting of the attention weights (appendix on rectangular
    matrices, application to Muon): per layer the q, k and v blocks of the
    d x 3d weight and the d x d projection each split into ``heads`` slices
    of d x d/heads; the MLP matrices stay whole."""
    out = []
    for _ in range(layers):
        out += [(d, d // heads)] * (4 * heads)
        out += [(d, 4 * d), (4 * d, d)]
    return out


def gpt2_heads(layers: int = 12, d: int = 768, heads: int = 12, first_seed: int = 5000) -> Workload:
    """GPT-2-small Muon step with per-head splitting: 576 slices of 768 x 64
    plus the 24 MLP matrices; spectra as in gpt2_small (s_i = 1/i +
    1e-3|N(0,1)|, unit Frobenius norm). Matrix j uses seed first_seed + j."""
    mats, svds = [], []
    for j, (m, n) in enumerate(gpt2_heads_shapes(layers, d, heads)):
        rng = np.random.default_rng(first_seed + j)
        sv_s = spectrum_gpt2(rng, min(m, n))
        sv_s = sv_s / np.linalg.norm(sv_s)
        sv = svd_matrix(rng, m, n, sv_s)
        mats.append(sv.G)
        svds.append(sv)
    return Workload("gpt2_small_per_head", mats, svds, 1e-3, 5, "bf16",
                    f"{layers} layers x ({4 * heads} heads of d x d/{heads}, d x 4d, 4d x d), d={d}")


def uneven_d1024(layers: int = 24, d: int = 1024, extra: int = 16,
                 shape_seed: int = 2) -> Workload:
    """24 layers of a d=1024 model plus ``extra`` matrices with m, n drawn
    uniformly from {128, 256, ..., 2048} (seed ``shape_seed``). Entries are
    N(0,1) plus a rank-8 spike (see gaussian_plus_spike); matrix j uses
    seed 1000 + j."""
    shapes = d1024_shapes(layers, d)
    srng = np.random.default_rng(shape_seed)
    choices = np.arange(128, 2049, 128)
    for _ in range(extra):
        shapes.append((int(srng.choice(choices)), int(srng.choice(choices))))
    mats = []
    for j, (m, n) in enumerate(shapes):
        rng = np.random.default_rng(1000 + j)
        mats.append(gaussian_plus_spike(rng, m, n))
    return Workload("uneven_d1024_plus16", mats, [None] * len(mats), 1e-3, 5, "bf16",
                    f"{layers} layers d={d} + {extra} random shapes, N(0,1)+rank-8 spike")


def large_dense(shapes: Sequence[Tuple[int, int]] = ((8192, 8192), (4096, 14336), (14336, 4096)),
                first_seed: int = 3) -> Workload:
    """Haar U, V with s log-uniform in [1e-4, 1], l = 1e-4, T = 6."""
    mats, svds = [], []
    for j, (m, n) in enumerate(shapes):
        rng = np.random.default_rng(first_seed + j)
        s = spectrum_loguniform(rng, min(m, n), 1e-4, 1.0)
        sv = svd_matrix(rng, m, n, s)
        mats.append(sv.G)
        svds.append(sv)
    return Workload("large_dense", mats, svds, 1e-4, 6, "bf16",
                    "Haar U,V; s log-uniform [1e-4,1]")


def ill_conditioned(shapes: Sequence[Tuple[int, int]] = ((2048, 2048), (4096, 1024)),
                    first_seed: int = 6, T: int = 12) -> Workload:
    """Haar U, V with s log-spaced in [1e-7, 1], l = 1e-7."""
    mats, svds = [], []
    for j, (m, n) in enumerate(shapes):
        rng = np.random.default_rng(first_seed + j)
        s = spectrum_logspaced(min(m, n), 1e-7, 1.0)
        sv = svd_matrix(rng, m, n, s)
        mats.append(sv.G)
        svds.append(sv)
    return Workload("ill_conditioned", mats, svds, 1e-7, T, "bf16x3",
                    "Haar U,V; s log-spaced [1e-7,1]")


def random_svd_case(seed: int, m: int, n: int, lo: float = 1e-3, hi: float = 1.0) -> SVDMatrix:
    """A small matrix with log-spaced spectrum in [lo, hi] (for parity tests)."""
    rng = np.random.default_rng(seed)
    return svd_matrix(rng, m, n, spectrum_logspaced(min(m, n), lo, hi))
