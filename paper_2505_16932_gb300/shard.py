"""Multi-GPU forms of the online stage.

polar_sharded: one model's Muon matrices over ranks. Polar factors of
different matrices are independent, so the only exchange is moving results:
whole matrices are assigned to ranks by longest processing time first on the
algorithmic flops T (3 s^2 L + s^3), each rank runs one grouped call on the
matrices it owns, and one all-gather of the flattened results gives every
rank every factor (NCCL on GPUs; gloo works for host tensors).

polar_split_long: one matrix cut along its long side over ranks. The squared
Frobenius norm and the Gram A = X X^T = sum_r X_r X_r^T are sums over the
ranks' blocks, B = b A + c A^2 is the same everywhere and X_r <- a X_r + B X_r
is local, so the exchange is one all-reduce of a scalar and one all-reduce
of the s x s FP32 Gram per polynomial step (Alg. 1 online stage, A on the
short side).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Optional, Sequence, Tuple


def step_flops(shape: Tuple[int, int], T: int = 1) -> float:
    m, n = shape
    s, L = min(m, n), max(m, n)
    return T * (3.0 * s * s * L + float(s) ** 3)


def assign(shapes: Sequence[Tuple[int, int]], world: int, T: int = 1) -> List[int]:
    """Owner rank of each matrix: LPT, ties to the lowest rank, deterministic."""
    if world < 1:
        raise ValueError("world >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-step_flops(shapes[i], T), i))
    heap = [(0.0, r) for r in range(world)]
    owners = [0] * len(shapes)
    for i in order:
        load, r = heapq.heappop(heap)
        owners[i] = r
        heapq.heappush(heap, (load + step_flops(shapes[i], T), r))
    return owners


def polar_sharded(Xs: Sequence, table, dtype: str = "bf16", group=None,
                  compute: Optional[Callable[[List], None]] = None):
    """In place on every rank's copy of Xs (same shapes and order on all ranks).

    ``compute`` overrides the per-rank computation (default: the library's
    pe_polar_batched); it receives the list of tensors this rank owns."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    shapes = [tuple(x.shape) for x in Xs]
    owners = assign(shapes, world, len(table))
    mine = [x for x, o in zip(Xs, owners) if o == rank]
    if compute is None:
        from . import pe_polar_batched

        def compute(xs):
            pe_polar_batched(xs, table, dtype)
    if mine:
        compute(mine)
    sizes = [0] * world
    for sh, o in zip(shapes, owners):
        sizes[o] += sh[0] * sh[1]
    cap = max(sizes) if sizes else 0
    if cap == 0:
        return Xs
    ref = Xs[0]
    send = torch.zeros(cap, dtype=ref.dtype, device=ref.device)
    off = 0
    for x in mine:
        send[off:off + x.numel()] = x.reshape(-1)
        off += x.numel()
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    pos = [0] * world
    for x, o in zip(Xs, owners):
        if o != rank:
            x.copy_(recv[o][pos[o]:pos[o] + x.numel()].view_as(x))
        pos[o] += x.numel()
    return Xs


def polar_split_long(X, table, short_is_rows: bool, dtype: str = "bf16", group=None, ops=None):
    """In place on this rank's block X of a matrix split along its long side.

    ``ops`` overrides the rank-local computation (default: the library's
    pe_split_* through paper_2505_16932_gb300.Split); it must provide
    sumsq(), set_norm(total), gram(t, A), step(t, A) and close(), with A an
    s x s tensor on X's device."""
    import torch
    import torch.distributed as dist

    if ops is None:
        from . import Split
        ops = Split(X, short_is_rows, table, dtype)
    s = X.shape[0] if short_is_rows else X.shape[1]
    T = len(table)
    try:
        tot = torch.tensor([ops.sumsq()], dtype=torch.float64, device=X.device)
        dist.all_reduce(tot, group=group)
        ops.set_norm(float(tot.item()))
        A = torch.empty((s, s), dtype=torch.float32 if X.is_cuda else torch.float64, device=X.device)
        for t in range(T):
            ops.gram(t, A)
            dist.all_reduce(A, group=group)
            ops.step(t, A)
    finally:
        ops.close()
    return X
