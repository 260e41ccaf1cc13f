"""Multi-rank host logic of the sharded batched call (gloo, world size 2, CPU).

The per-rank computation is the FP64 oracle here (no GPU), so the test checks
the assignment, the single all-gather exchange and that every rank ends with
the oracle's factor of every matrix; a rank that leaves before the exchange
makes the other rank's collective fail within its timeout instead of hanging.
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2505_16932_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_assign_lpt_balanced_and_deterministic():
    shapes = [(768, 2304), (768, 768), (768, 3072), (3072, 768)] * 12
    own = shard.assign(shapes, 4, T=5)
    assert own == shard.assign(shapes, 4, T=5)
    loads = [0.0] * 4
    for sh, o in zip(shapes, own):
        loads[o] += shard.step_flops(sh, 5)
    assert max(loads) / min(loads) < 1.05
    assert shard.assign([(5, 5)], 3) == [0]
    with pytest.raises(ValueError):
        shard.assign(shapes, 0)


def _worker(rank, world, port, mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    rng = np.random.default_rng(5)
    shapes = [(40, 24), (24, 60), (33, 33), (70, 20), (16, 16)]
    mats = [rng.standard_normal(s) for s in shapes]
    table, _ = O.optimal_composition(1e-2, 5, safety=1.01)
    Xs = [torch.from_numpy(m.copy()) for m in mats]

    def compute(xs):
        for x in xs:
            x.copy_(torch.from_numpy(O.polar_express(x.numpy(), table)))

    try:
        if mode == "dead" and rank == 1:
            return   # leaves before the exchange
        shard.polar_sharded(Xs, table, compute=compute)
        ok = all(np.allclose(x.numpy(), O.polar_express(m, table), atol=1e-12) for x, m in zip(Xs, mats))
        out[rank] = 1 if ok else 0
    except RuntimeError:
        out[rank] = 2
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.parametrize("world,mode", [(2, "ok"), (2, "dead"), (3, "ok")])
def test_sharded_gloo_ranks(world, mode):
    """Whole matrices over 2 or 3 gloo ranks (with 5 matrices, 3 ranks own
    uneven counts and byte totals, so the all-gather pads to the largest)."""
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", [-1] * world)
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        if p.is_alive():
            p.kill()
            pytest.fail("rank did not finish")
    if mode == "ok":
        assert list(out) == [1] * world
    else:
        assert out[0] == 2          # the survivor's collective failed, it did not hang


# ------------------------------------------------------ long-side split

class _NumpySplitOps:
    """Rank-local steps of the long-side split in FP64 (test stand-in for the
    library's pe_split_*): X_r is the rank's block in the short-side layout."""

    def __init__(self, X, short_is_rows, table):
        self.X = X                                   # torch float64 block, written at the end
        self.short_is_rows = short_is_rows
        self.Xr = X.numpy().copy() if short_is_rows else X.numpy().T.copy()
        self.table = table

    def sumsq(self):
        return float(np.sum(self.Xr * self.Xr))

    def set_norm(self, total):
        self.Xr = self.Xr / (1.01 * np.sqrt(total) + 1e-7)

    def gram(self, t, A):
        A.copy_(torch.from_numpy(self.Xr @ self.Xr.T))

    def step(self, t, A):
        a, b, c = self.table[t]
        An = A.numpy()
        self.Xr = a * self.Xr + (b * An + c * (An @ An)) @ self.Xr

    def close(self):
        self.X.copy_(torch.from_numpy(self.Xr if self.short_is_rows else self.Xr.T))


def _split_worker(rank, world, port, mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    table, _ = O.optimal_composition(1e-2, 5, safety=1.01)
    ok = True
    try:
        for short_is_rows, (m, n) in ((True, (24, 70)), (False, (64, 20))):
            G = np.random.default_rng(11).standard_normal((m, n))
            L = n if short_is_rows else m
            cuts = np.linspace(0, L, world + 1).astype(int)      # local extents may be < s
            lo, hi = cuts[rank], cuts[rank + 1]
            Gr = G[:, lo:hi] if short_is_rows else G[lo:hi, :]
            X = torch.from_numpy(Gr.copy())
            if mode == "dead" and rank == 1:
                return   # leaves before the first exchange
            shard.polar_split_long(X, table, short_is_rows, group=None, ops=_NumpySplitOps(X, short_is_rows, table))
            ref = O.polar_express(G, table)
            refr = ref[:, lo:hi] if short_is_rows else ref[lo:hi, :]
            ok = ok and np.allclose(X.numpy(), refr, atol=1e-12, rtol=0)
        out[rank] = 1 if ok else 0
    except RuntimeError:
        out[rank] = 2
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.parametrize("world,mode", [(2, "ok"), (3, "ok"), (2, "dead")])
def test_split_long_side_gloo(world, mode):
    """Long-side split over gloo ranks: one all-reduce of the squared norm and
    one of the Gram per step reproduce the FP64 iteration of the whole matrix
    on every rank's block, in both orientations, with local extents smaller
    than the short side; a rank that leaves makes the others' collective fail
    within the timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", [-1] * world)
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, mode, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        if p.is_alive():
            p.kill()
            pytest.fail("rank did not finish")
    if mode == "ok":
        assert list(out) == [1] * world
    else:
        assert out[0] == 2
