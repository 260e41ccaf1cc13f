"""GPU parity of the spectrum-aware initialisation (App. H, k = 1) through the C ABI.

* pe_spectrum_bound (power-method kernels on G) against the oracle's FP64
  power_bound on the same start vector, in both orientations, with row
  lengths that are and are not multiples of 4, and at a full GPT-2 MLP size;
  z never exceeds sigma_1.
* pe_polar_spectrum_aware (bound, host table, then the ordinary iteration)
  against the oracle's spectrum_aware_polar with the appendix's rule: FP32
  within 1e-5, BF16 and BF16x3 within 2e-2 relative Frobenius, l' within the
  propagated bound error; the gate option both ways; without a dominant
  singular value it is bitwise the plain call with T + 1 steps; the zero
  matrix stays zero.
* the appendix's power-law example (32 x 32, sigma_j = j^-5): with the cubic
  counted as an iteration, the FP32 GPU result is closer to U V^T than plain
  Polar Express at the same step count (by less than in FP64: the smallest
  singular values sit below FP32 resolution).
"""
import numpy as np
import pytest

import oracle as O
from oracle import spectrum_init as S

torch = pytest.importorskip("torch")
import paper_2505_16932_gb300 as pe  # noqa: E402
from paper_2505_16932_gb300 import build as B  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    pe.lib()
    yield
    torch.cuda.synchronize()


def _haar(rng, n, k):
    q, r = np.linalg.qr(rng.standard_normal((n, k)))
    return q * np.sign(np.diag(r))


def _gapped(seed, m, n, top=1.0, tail=(0.1, 1e-3)):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    U, V = _haar(rng, m, k), _haar(rng, n, k)
    s = np.concatenate([[top], np.geomspace(tail[0], tail[1], k - 1)])
    return (U * s) @ V.T, U, s, V


def dev(G):
    return torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,n,iters", [(96, 300, 8), (300, 96, 8), (130, 257, 5), (257, 130, 0), (1, 513, 3),
                                       (768, 3072, 10)])
def test_bound_matches_oracle(m, n, iters):
    G, U, s, V = _gapped(m * 7 + n, m, n)
    G32 = G.astype(np.float32).astype(np.float64)
    v0 = np.random.default_rng(1).standard_normal(min(m, n)).astype(np.float32)
    z, f = pe.pe_spectrum_bound(dev(G), v0, iters)
    X0, _ = O.normalise(G32)
    zr = S.power_bound(X0.T, v0.astype(np.float64), iters)
    # FP32 matrix-vector products against FP64: within the relative 1e-5 by
    # which the table shrinks z before use
    assert abs(z - zr) <= 1e-5 * zr, (z, zr)
    assert abs(f - np.linalg.norm(X0)) <= 1e-6 * f
    s1 = np.linalg.svd(X0, compute_uv=False)[0]
    assert z <= s1 * (1 + 1e-5)


@pytest.mark.parametrize("m,n", [(200, 520), (520, 200), (255, 255)])
def test_initialised_iteration_matches_oracle(m, n):
    """A gapped spectrum (sigma_2 / sigma_1 = 0.1, then log-spaced down to
    1e-3; l = 1e-3), the appendix's rule, against the oracle with the same
    z shrink the entry point applies to its FP32 bound (1e-5). l' = l / w
    depends on z through w = sqrt(f^2 - z^2) only, so its relative
    difference is the bound's relative difference times z^2 / w^2 (to first
    order; 4.5 here); the bound itself is within 1e-5 of the FP64 power
    method (test_bound_matches_oracle). T = 6 nearly converges, so the
    output moves by 6e-3 of the bound's relative change (T = 5: by 2.9x) and
    the FP32 bar is the iteration's own (3.5e-6 in a numpy FP32 run)."""
    G, _, _, _ = _gapped(m + 3 * n, m, n)
    G32 = G.astype(np.float32).astype(np.float64)
    v0 = np.random.default_rng(2).standard_normal(min(m, n)).astype(np.float32)
    ref, table, rinfo = S.spectrum_aware_polar(G32, 1e-3, 6, v0.astype(np.float64), 10, z_safety=1e-5)
    assert rinfo["applied"]
    z, w = rinfo["z"], rinfo["w"]
    for dtype, tol in (("fp32", 1e-5), ("bf16", 2e-2), ("bf16x3", 2e-2)):
        X = dev(G)
        info = pe.pe_polar_spectrum_aware(X, 1e-3, 6, v0, dtype, iters=10)
        pe.pe_sync_status()
        assert info["applied"]
        dz = (info["z"] - z) / z
        assert abs(dz) <= 1e-5
        dl = (info["l_after"] - rinfo["l_after"]) / rinfo["l_after"]
        pred = dz * z * z / (w * w)
        assert abs(dl - pred) <= 1e-3 * abs(pred) + 1e-9, (dl, pred)
        assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol, dtype


def test_gate_option_matches_oracle():
    """PE_SPECTRUM_GATE (not the appendix's rule): on a 1/i spectrum the
    intervals are disjoint, the appendix applies the cubic, and the gate
    keeps the plain composition; the entry point follows the oracle both ways
    and the gated call is bitwise the plain call with T + 1 steps."""
    rng = np.random.default_rng(8)
    m, n = 256, 640
    U, V = _haar(rng, m, m), _haar(rng, n, m)
    s = 1.0 / np.arange(1, m + 1)
    G = (U * s) @ V.T
    v0 = rng.standard_normal(m).astype(np.float32)
    for gate in (False, True):
        _, _, rinfo = S.spectrum_aware_polar(G.astype(np.float32).astype(np.float64), 1e-3, 4,
                                             v0.astype(np.float64), 10, z_safety=1e-5, gate=gate)
        X = dev(G)
        info = pe.pe_polar_spectrum_aware(X, 1e-3, 4, v0, "bf16", iters=10, gate=gate)
        pe.pe_sync_status()
        assert info["applied"] == rinfo["applied"] == (not gate)
    Y = dev(G)
    pe.pe_polar(Y, pe.pe_coeffs(5, 1e-3, 5, 1.01), "bf16")
    pe.pe_sync_status()
    assert torch.equal(X, Y)


def test_no_dominant_value_is_the_plain_call():
    rng = np.random.default_rng(6)
    G = rng.standard_normal((160, 400))
    v0 = rng.standard_normal(160).astype(np.float32)
    X = dev(G)
    info = pe.pe_polar_spectrum_aware(X, 1e-3, 5, v0, "bf16")
    assert not info["applied"]
    Y = dev(G)
    pe.pe_polar(Y, pe.pe_coeffs(5, 1e-3, 6, 1.01), "bf16")
    pe.pe_sync_status()
    assert torch.equal(X, Y)


def test_zero_matrix():
    X = torch.zeros(64, 96, device="cuda")
    z, f = pe.pe_spectrum_bound(X, np.ones(64), 5)
    assert z == 0.0 and f == 0.0
    info = pe.pe_polar_spectrum_aware(X, 1e-3, 4, np.ones(64), "fp32")
    pe.pe_sync_status()
    assert not info["applied"] and not torch.any(X != 0)


def test_power_law_example_converges_faster():
    rng = np.random.default_rng(0)
    n = 32
    U, V = _haar(rng, n, n), _haar(rng, n, n)
    s = np.arange(1, n + 1, dtype=np.float64) ** -5.0
    G = (U * s) @ V.T
    P = U @ V.T
    l = s[-1] / (1.01 * np.linalg.norm(s))
    v0 = rng.standard_normal(n).astype(np.float32)
    K = 12
    X = dev(G)
    info = pe.pe_polar_spectrum_aware(X, l, K - 1, v0, "fp32", iters=10)
    Y = dev(G)
    pe.pe_polar(Y, pe.pe_coeffs(5, l, K, 1.01), "fp32")
    pe.pe_sync_status()
    assert info["applied"]
    e_init = np.linalg.norm(X.cpu().numpy().astype(np.float64) - P, 2)
    e_plain = np.linalg.norm(Y.cpu().numpy().astype(np.float64) - P, 2)
    # FP32 resolves singular values only down to ~6e-8 of sigma_1 (the FP64
    # oracle pin of the same example shows a 50x gain at this step count);
    # measured on GB300 in FP32: 0.106 against 0.353
    assert e_init * 2 < e_plain, (e_init, e_plain)
