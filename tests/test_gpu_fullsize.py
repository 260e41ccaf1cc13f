"""Full-size parity on the workloads the benchmark times, through the C ABI.

* GPT-2-small Muon step (48 matrices, T = 5) in the benchmark's launch
  configuration (one grouped call, CUDA graph): every element of every
  matrix against the FP64 iteration in spectral form (exact for inputs
  drawn as U diag(s) V^T).
* Large dense (8192^2, 4096 x 14336, 14336 x 4096; l = 1e-4, T = 6): every
  element of the BF16 result against the FP64 iteration in spectral form;
  the BF16 and FP32 paths agree on the singular values of U1^T X V1 over the
  directions with s_i >= 1e-3 s_max, and those values follow the FP64 scalar
  composition p(x_i) of the oracle's table.
* Uneven batch with spikes (96 + 16 matrices, T = 5): every matrix against
  the dense FP64 iteration.
* Per-head splitting (576 head slices of 768 x 64 + 24 MLP matrices): every
  element of every matrix against the FP64 iteration in spectral form.
* Ill-conditioned spectra (2048^2, 4096 x 1024; l = 1e-7, T = 12): BF16x3 is
  closer to the FP64 iteration than BF16, on the restricted directions.
* Newton-Schulz quintic through the same kernels; the longest supported
  vector (1 x 2^20).
"""
import numpy as np
import pytest

import oracle as O
import synth

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


def dev(G):
    return torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()


def test_gpt2_small_full_size_elementwise():
    """All 48 matrices of the GPT-2-small step, every element, against the
    FP64 iteration in spectral form (U p(x) V^T: exact for inputs drawn as
    U diag(s) V^T), at the BF16 bar of 2e-2 relative Frobenius per matrix."""
    wl = synth.gpt2_small()
    tab = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    Xs = [dev(G) for G in wl.matrices]
    pe.pe_polar_batched(Xs, tab, "bf16")        # grouped, graph: the benchmark's configuration
    pe.pe_sync_status()
    worst = 0.0
    for X, sv, (m, n) in zip(Xs, wl.svd, wl.shapes):
        ref = O.polar_express_spectral(sv.U, sv.s, sv.V, tab)
        rel = O.rel_fro(X.cpu().numpy().astype(np.float64), ref)
        assert rel <= 2e-2, ((m, n), rel)
        worst = max(worst, rel)
    assert worst > 0.0


def _restricted_sv(X, U1, V1):
    C = U1.T.float() @ X.float() @ V1.float()      # FP32 products (TF32 off), FP32 SVD
    return torch.linalg.svdvals(C).double().cpu().numpy()


def test_large_dense_restricted_spectrum():
    shapes = [(8192, 8192), (4096, 14336), (14336, 4096)]
    T, l = 6, 1e-4
    tab = pe.pe_coeffs(5, l, T, 1.01)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    for m, n in shapes:
        k = min(m, n)
        U, _ = torch.linalg.qr(torch.randn(m, k, device="cuda", generator=gen, dtype=torch.float64))
        V, _ = torch.linalg.qr(torch.randn(n, k, device="cuda", generator=gen, dtype=torch.float64))
        e = torch.rand(k, device="cuda", generator=gen, dtype=torch.float64) * 4.0 - 4.0
        s = torch.sort(10.0 ** e, descending=True).values
        G = ((U * s) @ V.T).float().contiguous()
        keep = s >= 1e-3 * s[0]
        U1, V1 = U[:, keep].float(), V[:, keep].float()
        # oracle: the FP64 scalar composition at the normalised singular values
        sn = s.cpu().numpy()
        x = sn / (1.01 * np.sqrt(np.sum(sn * sn)) + 1e-7)
        px = np.sort(O.compose_scalar(x[keep.cpu().numpy()], tab))
        res = {}
        for path in ("bf16", "fp32"):
            X = G.clone()
            pe.pe_polar_batched([X], tab, path)
            pe.pe_sync_status()
            res[path] = np.sort(_restricted_sv(X, U1, V1))
            del X
        # both paths: kept directions follow p(x) of the oracle's table
        assert np.max(np.abs(res["fp32"] - px)) <= 2e-3, (m, n)
        assert np.max(np.abs(res["bf16"] - px)) <= 5e-2, (m, n)
        assert abs(np.max(np.abs(res["bf16"] - 1)) - np.max(np.abs(res["fp32"] - 1))) <= 2e-2
        del G, U, V, U1, V1
        torch.cuda.empty_cache()


def test_large_dense_bf16_every_element():
    """The benchmarked path on the large dense set (8192^2, 4096 x 14336,
    14336 x 4096; s log-uniform in [1e-4, 1], l = 1e-4, T = 6): every element
    of the BF16 result against the FP64 iteration in spectral form (U p(x)
    V^T from the oracle's scalar composition), at the BF16 bar of 2e-2
    relative Frobenius per matrix. (The spectral form is that of G before
    its FP32 rounding; on this spectrum the composition amplifies input
    perturbations about 10^3-fold in the directions below l, which puts the
    FP32 path at ~4e-5 from it and leaves the BF16 path's 16-bit master as
    the dominant term, ~1.5e-2.)"""
    shapes = [(8192, 8192), (4096, 14336), (14336, 4096)]
    T, l = 6, 1e-4
    tab = pe.pe_coeffs(5, l, T, 1.01)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    for m, n in shapes:
        k = min(m, n)
        U, _ = torch.linalg.qr(torch.randn(m, k, device="cuda", generator=gen, dtype=torch.float64))
        V, _ = torch.linalg.qr(torch.randn(n, k, device="cuda", generator=gen, dtype=torch.float64))
        e = torch.rand(k, device="cuda", generator=gen, dtype=torch.float64) * 4.0 - 4.0
        s = torch.sort(10.0 ** e, descending=True).values
        X = ((U * s) @ V.T).float().contiguous()
        pe.pe_polar_batched([X], tab, "bf16")     # one grouped call, graph: the benchmark's path
        pe.pe_sync_status()
        ref = O.polar_express_spectral(U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy(), tab)
        rel = O.rel_fro(X.double().cpu().numpy(), ref)
        assert rel <= 2e-2, ((m, n), rel)
        del X, U, V, ref
        torch.cuda.empty_cache()


def test_uneven_spike_batch_every_matrix():
    """The 112-matrix uneven batch (96 layer matrices + 16 random shapes,
    N(0,1) + rank-8 spike) in one grouped call: every matrix against the
    dense FP64 iteration on its FP32-cast input, at 2e-2."""
    wl = synth.uneven_d1024()
    tab = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    Xs = [dev(G) for G in wl.matrices]
    pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    for i, G in enumerate(wl.matrices):
        ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
        got = Xs[i].cpu().numpy().astype(np.float64)
        assert O.rel_fro(got, ref) <= 2e-2, (wl.shapes[i], O.rel_fro(got, ref))


@pytest.mark.parametrize("flags", [0, pe.PE_BATCH_PHASED])
def test_uneven_batch_bitwise_deterministic(flags):
    """Two runs of the 112-matrix batch give identical bits (catches races in
    the epilogue's shared-memory staging, which a small batch rarely hits)."""
    wl = synth.uneven_d1024()
    tab = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    outs = []
    for _ in range(2):
        pe.pe_release()
        Xs = [dev(G) for G in wl.matrices]
        pe.pe_polar_batched(Xs, tab, "bf16", flags=flags)
        pe.pe_sync_status()
        outs.append([X.cpu() for X in Xs])
    assert all(torch.equal(a, b) for a, b in zip(*outs))


def test_ill_conditioned_bf16x3_beats_bf16():
    wl = synth.ill_conditioned()
    tab = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    for G, sv in zip(wl.matrices, wl.svd):
        keep = sv.s >= 1e-3 * sv.s.max()
        U1 = torch.from_numpy(sv.U[:, keep]).cuda().float()
        V1 = torch.from_numpy(sv.V[:, keep]).cuda().float()
        x = sv.s / (1.01 * np.linalg.norm(sv.s) + 1e-7)
        px = np.sort(O.compose_scalar(x[keep], tab))
        err = {}
        for path in ("bf16", "bf16x3", "fp32"):
            X = dev(G)
            pe.pe_polar_batched([X], tab, path)
            pe.pe_sync_status()
            err[path] = float(np.max(np.abs(np.sort(_restricted_sv(X, U1, V1)) - px)))
        assert err["bf16x3"] < err["bf16"]
        assert err["bf16x3"] <= 5e-3 and err["fp32"] <= 5e-3, err


def test_newton_schulz_table_through_same_kernels():
    case = synth.random_svd_case(seed=4, m=640, n=1536, lo=0.05)
    tab = O.newton_schulz5_table(8)
    ref = O.polar_express_spectral(case.U, case.s, case.V, tab)
    for path, tol in (("fp32", 1e-5), ("bf16", 2e-2)):
        X = dev(case.G)
        pe.pe_polar(X, tab, path)
        pe.pe_sync_status()
        assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol


# The stated bars (FP32 1e-5, BF16 2e-2) on the longest supported vector:
# the FP32 Gram's reduction of length 2^20 runs as 256 chunks of 4096 summed
# in chunk order, so no accumulator sums more than 4096 products.
@pytest.mark.parametrize("path,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_longest_vector(path, tol):
    n = 1 << 20
    v = np.random.default_rng(1).standard_normal((1, n))
    tab = pe.pe_coeffs(5, 0.5, 4, 1.0)
    X = dev(v)
    pe.pe_polar(X, tab, path)
    pe.pe_sync_status()
    ref = O.polar_express_spectral(np.ones((1, 1)), np.array([np.linalg.norm(v)]),
                                   (v / np.linalg.norm(v)).T, tab)
    assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol


def test_gpt2_per_head_batch_every_element():
    """Per-head splitting (600 matrices: 576 head slices of 768 x 64, packed
    four to a descriptor, and the 24 MLP matrices) in one grouped call: every
    element of every matrix against the FP64 iteration in spectral form, at
    the BF16 bar of 2e-2 relative Frobenius per matrix."""
    wl = synth.gpt2_heads()
    tab = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    Xs = [dev(G) for G in wl.matrices]
    pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    worst = 0.0
    for i, (X, sv, (m, n)) in enumerate(zip(Xs, wl.svd, wl.shapes)):
        ref = O.polar_express_spectral(sv.U, sv.s, sv.V, tab)
        rel = O.rel_fro(X.cpu().numpy().astype(np.float64), ref)
        assert rel <= 2e-2, ((m, n), i, rel)
        worst = max(worst, rel)
    assert worst > 0.0
