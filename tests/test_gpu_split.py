"""Long-side split (pe_split_*) on one GPU.

Ranks are emulated one after another in this process (no kernel waits on
another): each block runs through the C ABI, the partial norms and Grams are
summed with torch between the calls, exactly what the all-reduces of
shard.polar_split_long do across GPUs.
* R = 1 gives the bits of pe_polar_batched with PE_BATCH_PHASED |
  PE_BATCH_NO_GRAPH (same kernels, same normalisation order).
* R = 3 (local extents smaller than the short side) matches the FP64
  iteration of the whole matrix: FP32 <= 1e-5, BF16 <= 2e-2.
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


def run_split(G, short_is_rows, table, dtype, R):
    L = G.shape[1] if short_is_rows else G.shape[0]
    s = G.shape[0] if short_is_rows else G.shape[1]
    cuts = np.linspace(0, L, R + 1).astype(int)
    blocks = []
    for r in range(R):
        lo, hi = cuts[r], cuts[r + 1]
        Gr = G[:, lo:hi] if short_is_rows else G[lo:hi, :]
        blocks.append(torch.from_numpy(np.ascontiguousarray(Gr, dtype=np.float32)).cuda())
    sp = [pe.Split(X, short_is_rows, table, dtype) for X in blocks]
    total = sum(h.sumsq() for h in sp)
    for h in sp:
        h.set_norm(total)
    A = torch.zeros((s, s), dtype=torch.float32, device="cuda")
    Ar = torch.zeros((s, s), dtype=torch.float32, device="cuda")
    for t in range(len(table)):
        A.zero_()
        for h in sp:
            h.gram(t, Ar)
            A += Ar
        for h in sp:
            h.step(t, A)
    for h in sp:
        h.close()
    out = torch.cat(blocks, dim=1 if short_is_rows else 0)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
@pytest.mark.parametrize("short_is_rows,shape", [(True, (384, 1000)), (False, (1000, 384))])
def test_split_one_rank_bitwise(dtype, short_is_rows, shape):
    G = np.random.default_rng(3).standard_normal(shape)
    tab = pe.pe_coeffs(5, 1e-3, 5, 1.01)
    got = run_split(G, short_is_rows, tab, dtype, 1)
    X = torch.from_numpy(G.astype(np.float32)).cuda()
    pe.pe_polar_batched([X], tab, dtype, flags=pe.PE_BATCH_PHASED | pe.PE_BATCH_NO_GRAPH)
    pe.pe_sync_status()
    assert np.array_equal(got, X.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("dtype,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
@pytest.mark.parametrize("short_is_rows", [True, False])
def test_split_three_ranks_vs_oracle(dtype, tol, short_is_rows):
    # log-spaced spectrum in [1e-3, 1]; L = 640 over 3 ranks
    # gives local extents 213/213/214 < s = 384
    case = synth.random_svd_case(seed=8, m=384, n=640, lo=1e-3)
    G = case.G if short_is_rows else case.G.T
    tab = pe.pe_coeffs(5, 1e-3, 6, 1.01)
    got = run_split(G, short_is_rows, tab, dtype, 3)
    pe.pe_sync_status()
    ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
    assert O.rel_fro(got, ref) <= tol


def test_split_call_order_enforced():
    X = torch.randn(128, 256, device="cuda")
    tab = pe.pe_coeffs(5, 1e-3, 2, 1.01)
    h = pe.Split(X, True, tab, "bf16")
    A = torch.zeros((128, 128), device="cuda")
    h.sumsq()
    with pytest.raises(pe.PolarExpressError):
        h.gram(0, A)          # before set_norm
    h.set_norm(1.0)
    with pytest.raises(pe.PolarExpressError):
        h.step(0, A)          # before gram(0)
    h.gram(0, A)
    with pytest.raises(pe.PolarExpressError):
        h.gram(1, A)          # step(0) missing
    h.close()
