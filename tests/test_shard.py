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


@pytest.mark.parametrize("mode", ["ok", "dead"])
def test_sharded_gloo_two_ranks(mode):
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", [-1, -1])
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        if p.is_alive():
            p.kill()
            pytest.fail("rank did not finish")
    if mode == "ok":
        assert list(out) == [1, 1]
    else:
        assert out[0] == 2          # the survivor's collective failed, it did not hang
