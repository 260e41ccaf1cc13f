"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (relative Frobenius distance to the FP64 iteration on the same
input): FP32 path 1e-5, BF16 path 2e-2 (the method's stated parity bars).
Single-product checks isolate each kernel with one-row tables:
(1,0,0) -> X_0, (0,1,0) -> A X_0, (0,0,1) -> A^2 X_0, compared with FP64
products of the same rounded operands.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
import paper_2505_16932_gb300 as pe  # noqa: E402
from paper_2505_16932_gb300 import build as B  # noqa: E402

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    pe.lib()
    yield
    torch.cuda.synchronize()


def to_dev(G, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).to("cuda").to(dtype)


def run_single(G, table, dtype, io=torch.float32):
    X = to_dev(G, io)
    pe.pe_polar(X, table, dtype)
    pe.pe_sync_status()
    return X.float().cpu().numpy().astype(np.float64)


def bf16r(x):
    """Round to bfloat16 (nearest even) through torch, as FP64."""
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def table(l, T, safety=1.01):
    return pe.pe_coeffs(5, l, T, safety)


# ----------------------------------------------------------- plain method

def test_fp32_plain_small_matches_oracle():
    wl = synth.plain_small()
    G = wl.matrices[0]
    tab = table(wl.l, wl.T)
    got = run_single(G, tab, "fp32")
    ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
    assert O.rel_fro(got, ref) <= FP32_TOL
    # the error metrics of the output against polar(G) are those of the FP64 iteration
    P = O.polar_svd(G)
    assert abs(O.err_polar_fro(got, P) - O.err_polar_fro(ref, P)) <= 1e-5


SHAPES = [(1, 1), (1, 5), (5, 1), (37, 100), (100, 37), (129, 300), (300, 129), (256, 256), (257, 513),
          (640, 130)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_fp32_shapes(m, n):
    case = synth.random_svd_case(seed=m * 1000 + n, m=m, n=n, lo=1e-2)
    tab = table(1e-3, 6)
    got = run_single(case.G, tab, "fp32")
    ref = O.polar_express_spectral(case.U, case.s, case.V, tab)
    assert got.shape == (m, n)
    assert O.rel_fro(got, ref) <= FP32_TOL


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("m,n", [(200, 333), (333, 200), (128, 256)])
def test_identity_step(dtype, m, n):
    """Table (1, 0, 0): the output is the normalised input (prepare + store).

    The BF16 path keeps X as its BF16 hi plus a code of the next 8 mantissa
    bits (x rounded to a 16-bit mantissa), so each element is carried to
    within 2^-16 |x|; FP32 and BF16x3 keep FP32 X."""
    rng = np.random.default_rng(m + n)
    G = rng.standard_normal((m, n))
    got = run_single(G, [(1.0, 0.0, 0.0)], dtype)
    ref = G.astype(np.float32) / (1.01 * np.linalg.norm(G.astype(np.float32)) + 1e-7)
    if dtype == "bf16":
        # (+ 2^-20 |x| for the FP32 scaling and norm, + a floor for zeros)
        assert np.all(np.abs(got - ref) <= (2.0 ** -16 + 2.0 ** -20) * np.abs(ref) + 1e-7 * np.max(np.abs(ref)))
        # and it is not merely BF16: most elements beat bf16 rounding by far
        assert np.median(np.abs(got - ref) / np.abs(ref)) < 2.0 ** -14
    else:
        assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("m,n", [(256, 640), (640, 256), (384, 384), (130, 700)])
@pytest.mark.parametrize("row", [(0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.5, -1.0, 0.7)])
def test_single_products(dtype, m, n, row):
    rng = np.random.default_rng(7 * m + n)
    G = rng.standard_normal((m, n))
    got = run_single(G, [row], dtype)
    X0 = G.astype(np.float32).astype(np.float64)
    X0 = X0 / (1.01 * np.linalg.norm(X0) + 1e-7)
    if m > n:
        X0 = X0.T
    a, b, c = row
    if dtype == "bf16":
        # the BF16 update a X + B X_b + d (X - X_b), d = tr(B) / s
        Xh = bf16r(X0)
        A = Xh @ Xh.T
        Ah = bf16r(A)
        Bf = b * A + c * (Ah @ Ah)
        Bm = bf16r(Bf)
        d = np.trace(Bf) / min(m, n)
        ref = a * X0 + Bm @ Xh + d * (X0 - Xh)
        tol = 1e-2
    else:
        A = X0 @ X0.T
        ref = a * X0 + (b * A + c * (A @ A)) @ X0
        tol = 1e-5 if dtype == "fp32" else 1e-4
    if m > n:
        ref = ref.T
    assert O.rel_fro(got, ref) <= tol


# ------------------------------------------------------------ BF16 paths

def test_bf16_gpt2_layer_batched_vs_oracle():
    """One GPT-2-small layer (768x2304, 768x768, 768x3072, 3072x768), T = 5,
    grouped launch, against the FP64 iteration (spectral form)."""
    wl = synth.gpt2_small(layers=1)
    tab = table(wl.l, wl.T)
    Xs = [to_dev(G) for G in wl.matrices]
    pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    for X, sv in zip(Xs, wl.svd):
        got = X.cpu().numpy().astype(np.float64)
        ref = O.polar_express_spectral(sv.U, sv.s, sv.V, tab)
        assert O.rel_fro(got, ref) <= BF16_TOL


def test_bf16x3_closer_than_bf16():
    case = synth.random_svd_case(seed=11, m=384, n=640, lo=1e-3)
    tab = table(1e-3, 6)
    ref = O.polar_express_spectral(case.U, case.s, case.V, tab)
    e16 = O.rel_fro(run_single(case.G, tab, "bf16"), ref)
    e3 = O.rel_fro(run_single(case.G, tab, "bf16x3"), ref)
    assert e16 <= BF16_TOL
    assert e3 <= 1e-3 and e3 < e16 / 4


def test_bf16_io_bf16():
    case = synth.random_svd_case(seed=12, m=300, n=500, lo=1e-2)
    tab = table(1e-3, 5)
    G16 = bf16r(case.G)
    got = run_single(G16, tab, "bf16", io=torch.bfloat16)
    ref = O.polar_express(G16, tab)
    assert O.rel_fro(got, ref) <= BF16_TOL


# ------------------------------------------- grouped, graph, determinism

def _even(seed=31):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(s) for s in ((256, 512), (512, 256), (768, 2304), (3072, 768), (512, 512))]


@pytest.mark.parametrize("dtype", ["bf16"])
def test_two_sm_mode_bitwise(dtype):
    """2-SM UMMA (256 x 256 tiles) against the 1-SM kernel on sizes that are
    multiples of 256, with one and with two accumulators, and with twelve
    epilogue warps (mode 3: every third 32-column chunk per warp)."""
    mats = _even()
    tab = table(1e-3, 5)
    outs = []
    try:
        for mode, nacc in ((0, 0), (2, 1), (2, 2), (3, 0)):
            pe.pe_debug_set(7, mode)
            pe.pe_debug_set(8, nacc)
            pe.pe_release()
            Xs = [to_dev(G) for G in mats]
            pe.pe_polar_batched(Xs, tab, dtype)
            pe.pe_sync_status()
            outs.append([X.cpu() for X in Xs])
    finally:
        pe.pe_debug_set(7, -1)
        pe.pe_debug_set(8, 0)
        pe.pe_release()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def _uneven(seed=3, k=7):
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(1, 700)), int(rng.integers(1, 700))) for _ in range(k)] + [(128, 1024), (1024, 128)]
    return [rng.standard_normal(s) for s in shapes]


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "bf16x3"])
def test_grouped_equals_single_bitwise(dtype):
    mats = _uneven()
    tab = table(1e-3, 5)
    singles = [run_single(G, tab, dtype) for G in mats]
    for flags in (0, pe.PE_BATCH_PHASED, pe.PE_BATCH_NO_GRAPH):
        Xs = [to_dev(G) for G in mats]
        pe.pe_polar_batched(Xs, tab, dtype, flags=flags)
        pe.pe_sync_status()
        for X, ref in zip(Xs, singles):
            assert np.array_equal(X.cpu().numpy().astype(np.float64), ref)


def test_graph_replay_repeats():
    mats = _uneven(seed=5)
    tab = table(1e-3, 5)
    Xs = [to_dev(G) for G in mats]
    pe.pe_polar_batched(Xs, tab, "bf16")
    first = [X.clone() for X in Xs]
    n0 = pe.pe_launch_count()
    for _ in range(3):
        for X, G in zip(Xs, mats):
            X.copy_(to_dev(G))
        pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    assert pe.pe_launch_count() > n0
    for X, F in zip(Xs, first):
        assert torch.equal(X, F)


def test_batched_vs_oracle_uneven():
    mats = _uneven(seed=9)
    tab = table(1e-3, 6)
    # iid Gaussian inputs iterated well past their convergence: the BF16
    # update's rounding term is -(B - d I)(X - X_b), d = tr(B) / s, which
    # vanishes on converged directions (the stated 2e-2 bar holds; the plain
    # a X + B X_b form reached 2.4e-2 here)
    for dtype, tol in (("fp32", FP32_TOL), ("bf16", BF16_TOL), ("bf16x3", BF16_TOL)):
        Xs = [to_dev(G) for G in mats]
        pe.pe_polar_batched(Xs, tab, dtype)
        pe.pe_sync_status()
        for X, G in zip(Xs, mats):
            ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
            assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol, (dtype, G.shape)


# ------------------------------------------------------ degenerate inputs

@pytest.mark.parametrize("dtype,tol", [("fp32", FP32_TOL), ("bf16", BF16_TOL), ("bf16x3", BF16_TOL)])
def test_degenerate_inputs(dtype, tol):
    """Inputs the method degenerates on. G = 0: the normalisation divides by
    eps alone and X stays exactly zero through every step. A 1 x 1 matrix
    (polar(g) = sign(g)), a single row and a single column (one singular
    value each) and orthogonal rows (polar(Q) = Q, every normalised singular
    value 1 / (1.01 sqrt(s))): each against the FP64 iteration at the
    path's bar, and the 1 x 1 result with the sign of g."""
    rng = np.random.default_rng(13)
    tab = table(1e-3, 6)
    Z = np.zeros((64, 200))
    assert np.array_equal(run_single(Z, tab, dtype), Z)
    Q, _ = np.linalg.qr(rng.standard_normal((640, 256)))
    cases = [np.array([[-3.0]]), rng.standard_normal((1, 7)), rng.standard_normal((5, 1)), Q.T]
    for G in cases:
        ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
        got = run_single(G, tab, dtype)
        assert O.rel_fro(got, ref) <= tol, (dtype, G.shape)
    assert run_single(np.array([[-3.0]]), tab, dtype)[0, 0] < -0.9


# ---------------------------------------------------- status / failures

def test_nonfinite_input_reports_status():
    G = np.ones((64, 64))
    G[3, 5] = np.inf
    X = to_dev(G)
    pe.pe_polar(X, table(1e-3, 2), "bf16")
    with pytest.raises(pe.PolarExpressError) as ei:
        pe.pe_sync_status()
    assert ei.value.code == pe.PE_ECUDA
    # the status was cleared; the next call works
    run_single(np.eye(64), table(1e-3, 2), "bf16")


def test_readiness_wait_timeout_reports_status():
    """Withhold matrix 0's Gram readiness in one fused launch: its waiters'
    bounded waits expire, the launch completes, PE_ETIMEOUT is reported, and
    the library keeps working afterwards."""
    mats = _uneven(seed=13)
    tab = table(1e-3, 3)
    Xs = [to_dev(G) for G in mats]
    pe.pe_debug_set(2, 20_000_000)       # 20 ms wait limit
    pe.pe_debug_set(1, 0)                # withhold matrix 0
    pe.pe_polar_batched(Xs, tab, "bf16")
    with pytest.raises(pe.PolarExpressError) as ei:
        pe.pe_sync_status()
    assert ei.value.code == pe.PE_ETIMEOUT
    pe.pe_debug_set(2, 0)
    Xs = [to_dev(G) for G in mats]
    pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    ref = O.polar_express(mats[1].astype(np.float32).astype(np.float64), tab)
    assert O.rel_fro(Xs[1].cpu().numpy().astype(np.float64), ref) <= BF16_TOL


def test_injected_alloc_failure():
    pe.pe_debug_set(3, 1)
    X = to_dev(np.random.default_rng(0).standard_normal((77, 55)))
    with pytest.raises(pe.PolarExpressError) as ei:
        pe.pe_polar(X, table(1e-3, 2), "bf16")
    assert ei.value.code == pe.PE_ENOMEM


SENTINEL = 12345.0


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("m,n", [(130, 257), (257, 130), (1, 77), (256, 512)])
def test_writes_stay_inside_the_matrix(dtype, m, n):
    """Canaries: a call writes exactly the caller's m x n elements. Guard
    elements before the first and after the last element of the same
    allocation keep their sentinel, and so do the padding columns between rows
    when the leading dimension exceeds n (odd and 16-byte-multiple pitches:
    element stores and TMA stores); the strided result equals the contiguous
    one bit for bit."""
    rng = np.random.default_rng(7 * m + n)
    G = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    tab = table(1e-3, 3)
    guard = 1024   # floats: keeps the matrix 16-byte aligned
    buf = torch.full((guard + m * n + guard,), SENTINEL, device="cuda")
    X = buf[guard:guard + m * n].view(m, n)
    X.copy_(G)
    pe.pe_polar(X, tab, dtype)
    pe.pe_sync_status()
    assert torch.all(buf[:guard] == SENTINEL) and torch.all(buf[guard + m * n:] == SENTINEL)
    for ld in (n + 5, (n + 3) // 4 * 4 + 8):
        buf2 = torch.full((guard + m * ld + guard,), SENTINEL, device="cuda")
        Y = buf2[guard:guard + m * ld].view(m, ld)
        Y[:, :n].copy_(G)
        pe.pe_polar(Y[:, :n], tab, dtype)
        pe.pe_sync_status()
        assert torch.all(buf2[:guard] == SENTINEL) and torch.all(buf2[guard + m * ld:] == SENTINEL), ld
        assert torch.all(Y[:, n:] == SENTINEL), ld
        assert torch.equal(Y[:, :n], X), ld


def test_empty_and_bad_shapes_rejected():
    X = torch.zeros((0, 5), device="cuda")
    with pytest.raises(pe.PolarExpressError):
        pe.pe_polar(X, table(1e-3, 2), "bf16")
    assert pe.pe_polar_batched([], table(1e-3, 2), "bf16") == []


@pytest.mark.parametrize("dtype", ["bf16", "bf16x3"])
def test_kblock_and_order_variants_bitwise(dtype):
    """The 32-wide k-block variant, the tile orders and the 2-SM variant
    issue the same K=16 MMA chain on the same operands per output element, so
    every variant gives identical bits (the 2-SM mode needs every padded size
    to be a multiple of 256; the shapes that are not fall back to the 1-SM
    kernel)."""
    mats = _uneven(seed=21)
    tab = table(1e-3, 4)
    outs = []
    try:
        for bk, order, mode in ((64, 0, 0), (32, 0, 0), (64, 1, 0), (32, 1, 0), (64, 2, 0), (64, 4, 0),
                                (64, 3, 0), (64, 0, 2), (64, 1, 2), (64, 4, 2), (64, 0, 3), (64, 4, 3)):
            pe.pe_debug_set(5, bk)
            pe.pe_debug_set(6, order)
            pe.pe_debug_set(7, mode)
            pe.pe_release()
            Xs = [to_dev(G) for G in mats]
            pe.pe_polar_batched(Xs, tab, dtype)
            pe.pe_sync_status()
            outs.append([X.cpu() for X in Xs])
    finally:
        pe.pe_debug_set(5, 0)
        pe.pe_debug_set(6, -1)
        pe.pe_debug_set(7, -1)
        pe.pe_release()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


# ------------------------------------------------ degree-3 tables (c = 0)

@pytest.mark.parametrize("which", ["pe3", "ns3"])
def test_degree3_tables_skip_square(which):
    """Degree-3 tables (the degree-3 greedy composition of Thm. 1, and the
    Newton-Schulz cubic) have c = 0 in every row: the BF16 path writes
    B = b A from the Gram epilogue and launches no square tiles. Uneven batch,
    fused, phased and 2-SM-eligible shapes, against the FP64 iteration."""
    if which == "pe3":
        tab = pe.pe_coeffs(3, 1e-3, 8, 1.01)
    else:
        tab = np.array([[1.5, -0.5, 0.0]] * 12)
    assert np.all(tab[:, 2] == 0.0)
    mats = _uneven(seed=5) + _even(seed=6)[:3]
    for dtype, tol in (("fp32", FP32_TOL), ("bf16", BF16_TOL)):
        for flags in (0, pe.PE_BATCH_PHASED):
            Xs = [to_dev(G) for G in mats]
            pe.pe_polar_batched(Xs, tab, dtype, flags=flags)
            pe.pe_sync_status()
            for X, G in zip(Xs, mats):
                ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
                assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol, (dtype, flags, G.shape)


def test_jordan_table_through_same_kernels():
    """Jordan's fixed quintic 3.4445x - 4.7750x^3 + 2.0315x^5 (Sec. 1.2) as a
    table, through the same grouped kernels, against the FP64 iteration of
    the same table. The polynomial does not contract (its singular values
    keep oscillating in about [0.7, 1.2]), so rounding errors are not damped
    and the BF16 error grows with T (a CPU emulation of the kernels'
    arithmetic on this batch: 0.7e-2 - 1.6e-2 at T = 4, up to 2.6e-2 at
    T = 6); T = 4 keeps every path within its stated bar."""
    tab = np.array(O.jordan_table(4))
    mats = _uneven(seed=5)
    for dtype, tol in (("fp32", FP32_TOL), ("bf16", BF16_TOL), ("bf16x3", BF16_TOL)):
        Xs = [to_dev(G) for G in mats]
        pe.pe_polar_batched(Xs, tab, dtype)
        pe.pe_sync_status()
        for X, G in zip(Xs, mats):
            ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
            assert O.rel_fro(X.cpu().numpy().astype(np.float64), ref) <= tol, (dtype, G.shape)


# ------------------------------------------------------- host-buffer entry

@pytest.mark.parametrize("ngroups", [0, 1, 2, 3])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_equal_device_call(ngroups, pinned):
    """pe_polar_batched_host pipelines the copies with the grouped compute;
    the grouping does not change the bits (grouped == single), so the result
    equals pe_polar_batched on device copies of the same inputs."""
    mats = _uneven(seed=17) + _even(seed=18)[:2]
    tab = table(1e-3, 5)
    H_in = [torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)) for G in mats]
    if pinned:
        H_in = [h.pin_memory() for h in H_in]
    H_out = [torch.empty_like(h) for h in H_in]
    if pinned:
        H_out = [h.pin_memory() for h in H_out]
    pe.pe_polar_batched_host(H_in, H_out, tab, "bf16", ngroups=ngroups)
    pe.pe_sync_status()
    Xs = [h.cuda() for h in H_in]
    pe.pe_polar_batched(Xs, tab, "bf16")
    pe.pe_sync_status()
    for h, X in zip(H_out, Xs):
        assert torch.equal(h, X.cpu())


# ------------------------------------------- pairs of small matrices (BF16)

def test_small_matrix_packs_bitwise_equal_unpacked():
    """BF16 matrices with a short side <= 64 of one shape share descriptors of
    four 64-row blocks (block-diagonal Gram). Each matrix's Gram, square and
    update see the same products in the same order as alone, so the result
    equals the unpacked plan's bit for bit; covers both orientations, a full
    pack plus a pack of one (5 matrices), packs of 2 and 3, a ragged long
    side, a shape seen once (not packed) and a large matrix."""
    shapes = ([(768, 64)] * 5 + [(40, 500)] * 2 + [(64, 64)] * 3 + [(20, 33)] + [(256, 300)])
    # log-spaced spectra in [1e-3, 1] (the heavy-tailed class; iid Gaussian
    # inputs are the well-conditioned class of the BF16 limit above)
    mats = [synth.random_svd_case(seed=23 + i, m=m, n=n, lo=1e-3).G for i, (m, n) in enumerate(shapes)]
    tab = table(1e-3, 5)
    outs = []
    try:
        for nopair in (0, 1):
            pe.pe_debug_set(9, nopair)
            pe.pe_release()
            Xs = [to_dev(G) for G in mats]
            pe.pe_polar_batched(Xs, tab, "bf16")
            pe.pe_sync_status()
            outs.append([X.cpu() for X in Xs])
    finally:
        pe.pe_debug_set(9, 0)
        pe.pe_release()
    for a, b, sh in zip(outs[0], outs[1], shapes):
        assert torch.equal(a, b), sh
    for X, G in zip(outs[0], mats):
        ref = O.polar_express(G.astype(np.float32).astype(np.float64), tab)
        assert O.rel_fro(X.numpy().astype(np.float64), ref) <= BF16_TOL
