"""Fused Muon step (pe_muon_batched): M <- beta M + (1 - beta) G,
W <- W - lr polar(M) (Sec. 2.1), through the C ABI, against the FP64 oracle.

* The momentum is exact FP32 arithmetic: fma(beta, M, fl((1 - beta) G)),
  checked to 1 ulp (the reference is formed in FP64 and rounded once more).
* With W = 0 the weight update is -lr X_T exactly (lr a power of two), so
  X_T is checked against the FP64 iteration of the new M at the parity bars
  (FP32 1e-5, BF16 2e-2).
* With a random W, (W - W') / lr is checked at the BF16 bar.
* The first call tunes the plan without touching M or W; a second call
  (graph replay) accumulates the momentum once more.
Shapes cover both orientations and widths that are not a multiple of 4 (no
TMA for the weight update: read-modify-write stores).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
import paper_2505_16932_gb300 as pe  # noqa: E402
from paper_2505_16932_gb300 import build as B  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(256, 640), (640, 256), (300, 130), (130, 301)]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    pe.lib()
    yield
    torch.cuda.synchronize()


def _mom_ref(beta, M, G):
    b = np.float32(beta)
    omb = np.float32(np.float32(1.0) - b)
    t = (omb.astype(np.float64) * G.astype(np.float64)).astype(np.float32)   # fl((1 - beta) G)
    return (b.astype(np.float64) * M.astype(np.float64) + t.astype(np.float64)).astype(np.float32)


def _inputs(seed):
    # gradient and earlier momentum both with log-spaced spectra in [1e-3, 1]
    # (the heavy-tailed class of the Muon workloads; a momentum of iid noise
    # would be the well-conditioned class, see the BF16 limit in test_gpu_parity)
    Gs, Ms = [], []
    for i, (m, n) in enumerate(SHAPES):
        Gs.append(synth.random_svd_case(seed=seed + i, m=m, n=n, lo=1e-3).G.astype(np.float32))
        Ms.append((0.5 * synth.random_svd_case(seed=seed + 100 + i, m=m, n=n, lo=1e-3).G).astype(np.float32))
    return Gs, Ms


def _ulps(a, b):
    return np.max(np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64)))


@pytest.mark.parametrize("dtype,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_muon_zero_weights(dtype, tol):
    beta, lr = 0.9, 0.5
    tab = pe.pe_coeffs(5, 1e-3, 6, 1.01)
    Gs, Ms = _inputs(20)
    Gd = [torch.from_numpy(G).cuda() for G in Gs]
    Md = [torch.from_numpy(M).cuda() for M in Ms]
    Wd = [torch.zeros_like(G) for G in Gd]
    pe.pe_muon_batched(Wd, Gd, Md, beta, lr, tab, dtype)
    pe.pe_sync_status()
    for G, M, Mg, Wg in zip(Gs, Ms, Md, Wd):
        M1 = _mom_ref(beta, M, G)
        assert _ulps(Mg.cpu().numpy(), M1) <= 1
        ref = O.polar_express(M1.astype(np.float64), tab)
        X = -Wg.cpu().numpy().astype(np.float64) / lr
        assert O.rel_fro(X, ref) <= tol, (dtype, G.shape)


def test_muon_random_weights_two_calls():
    beta, lr = 0.9, 0.02
    tab = pe.pe_coeffs(5, 1e-3, 5, 1.01)
    Gs, Ms = _inputs(40)
    rng = np.random.default_rng(41)
    Ws = [rng.standard_normal(G.shape).astype(np.float32) for G in Gs]
    Gd = [torch.from_numpy(G).cuda() for G in Gs]
    Md = [torch.from_numpy(M).cuda() for M in Ms]
    Wd = [torch.from_numpy(W).cuda() for W in Ws]
    M_host = [M.copy() for M in Ms]
    W_host = [W.astype(np.float64) for W in Ws]
    for call in range(2):
        if call == 1:   # new gradients in the same buffers: the cached plan (graph) is replayed
            for i, G in enumerate(Gs):
                Gs[i] = (G[::-1, ::-1] * 0.7).copy()
                Gd[i].copy_(torch.from_numpy(Gs[i]))
        pe.pe_muon_batched(Wd, Gd, Md, beta, lr, tab, "bf16")
        pe.pe_sync_status()
        for i, G in enumerate(Gs):
            M_host[i] = _mom_ref(beta, M_host[i], G)
            assert _ulps(Md[i].cpu().numpy(), M_host[i]) <= 1
            ref = O.polar_express(M_host[i].astype(np.float64), tab)
            Wn = Wd[i].cpu().numpy().astype(np.float64)
            assert O.rel_fro((W_host[i] - Wn) / lr, ref) <= 2e-2, (call, G.shape)
            W_host[i] = Wn


def test_muon_argument_errors():
    X = torch.zeros(8, 8, device="cuda")
    tab = pe.pe_coeffs(5, 1e-3, 2, 1.01)
    with pytest.raises(pe.PolarExpressError):
        pe.pe_muon_batched([X], [X], [X], 1.5, 0.1, tab)            # beta outside [0, 1]
    with pytest.raises(pe.PolarExpressError):
        pe.pe_muon_batched([X], [X, X], [X], 0.9, 0.1, tab)         # list lengths
    with pytest.raises(pe.PolarExpressError):
        pe.pe_muon_batched([X], [X.bfloat16()], [X], 0.9, 0.1, tab)  # dtype
