"""IJK-partitioned multi-process driver pieces (Sec. III.A.1-III.A.3).

``IJKPlan`` wraps the library's host planner (``rccsdt_ijk_plan_*``): which rank
owns each stored block of compact T3/R3, and the batches of the step (v)
exchange.  ``gather_batches`` runs that exchange over ``torch.distributed`` (gloo
on CPU ranks, NCCL on GPUs): one all-gather per batch, the next batch in flight
while the caller contracts the current one (the double buffer of Sec. III.A.3),
so every T3 element crosses the network once per cycle.  ``allreduce_sum_`` is the
small reduction of steps (iii) and (vii).

This module moves data only: the contractions, norms and updates on each rank are
the caller's (the library's kernels on a GPU rank).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .binding import OK, RccsdtError


class IJKPlan:
    """Ownership and exchange batches of the stored blocks i <= j <= k for `nranks`
    processes; `batch_triples` is the mean number of blocks per batch; `cost`
    (float64[n3]) replaces the library's per-block cost model."""

    def __init__(self, lib, o: int, v: int, nranks: int, batch_triples: int, cost=None):
        self.lib, self.o, self.v, self.nranks = lib, o, v, nranks
        h = C.c_void_p()
        cbuf = None
        if cost is not None:
            cbuf = np.ascontiguousarray(cost, dtype=np.float64)
        st = lib.rccsdt_ijk_plan_create(o, v, nranks, batch_triples,
                                        cbuf.ctypes.data if cbuf is not None else None, C.byref(h))
        if st != OK:
            raise RccsdtError(st, "rccsdt_ijk_plan_create failed")
        self.h = h
        info = np.zeros(6, dtype=np.int64)
        lib.rccsdt_ijk_plan_info(h, info.ctypes.data)
        self.n3, _, self.nbatches, self.max_owned, self.max_batch, self.max_send = (int(x) for x in info)

    @staticmethod
    def default_costs(lib, o: int, v: int) -> np.ndarray:
        out = np.zeros(o * (o + 1) * (o + 2) // 6)
        st = lib.rccsdt_ijk_block_costs(o, v, out.ctypes.data)
        if st != OK:
            raise RccsdtError(st, "rccsdt_ijk_block_costs failed")
        return out

    def owners(self) -> np.ndarray:
        out = np.zeros(self.n3, dtype=np.int32)
        self.lib.rccsdt_ijk_plan_owners(self.h, out.ctypes.data)
        return out

    def local(self, rank: int) -> np.ndarray:
        n = C.c_int()
        st = self.lib.rccsdt_ijk_plan_local(self.h, rank, None, C.byref(n))
        if st != OK:
            raise RccsdtError(st, "rccsdt_ijk_plan_local failed")
        out = np.zeros(n.value, dtype=np.int32)
        self.lib.rccsdt_ijk_plan_local(self.h, rank, out.ctypes.data, C.byref(n))
        return out

    def batch(self, b: int):
        """(counts[nranks], blocks grouped by owner in rank order) of batch b."""
        counts = np.zeros(self.nranks, dtype=np.int32)
        st = self.lib.rccsdt_ijk_plan_batch(self.h, b, counts.ctypes.data, None)
        if st != OK:
            raise RccsdtError(st, "rccsdt_ijk_plan_batch failed")
        blocks = np.zeros(int(counts.sum()), dtype=np.int32)
        self.lib.rccsdt_ijk_plan_batch(self.h, b, counts.ctypes.data, blocks.ctypes.data)
        return counts, blocks

    def work(self):
        """(rank_cost[nranks], batch_work[nbatches, nranks])."""
        rc = np.zeros(self.nranks)
        bw = np.zeros((self.nbatches, self.nranks))
        self.lib.rccsdt_ijk_plan_work(self.h, rc.ctypes.data, bw.ctypes.data)
        return rc, bw

    def close(self):
        if self.h:
            self.lib.rccsdt_ijk_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather_batches(plan: IJKPlan, rank: int, local_t3, consume, group=None, overlap: bool = True):
    """Step (v)'s exchange.  `local_t3` is a torch tensor [len(plan.local(rank)), ...]
    holding this rank's blocks in storage order.  For each batch b, every rank's
    blocks of the batch are gathered onto every rank (one all-gather, each rank's
    share padded to the batch's largest share) and `consume(b, blocks, data)` is
    called with the batch's block indices (grouped by owner in rank order) and a
    tensor [len(blocks), ...] of their values.  With `overlap`, the all-gather of
    batch b + 1 is issued before batch b is consumed (two receive buffers).
    Returns the number of blocks this rank sent."""
    import torch
    import torch.distributed as dist

    mine = {int(b): q for q, b in enumerate(plan.local(rank))}
    shape = tuple(local_t3.shape[1:])
    sent = 0

    def issue(b):
        nonlocal sent
        counts, blocks = plan.batch(b)
        width = int(counts.max())
        off = int(counts[:rank].sum())
        own = blocks[off:off + int(counts[rank])]
        send = torch.zeros((width,) + shape, dtype=local_t3.dtype, device=local_t3.device)
        if len(own):
            idx = torch.as_tensor([mine[int(x)] for x in own], device=local_t3.device)
            send[:len(own)] = local_t3.index_select(0, idx)
        sent += len(own)
        recv = [torch.empty_like(send) for _ in range(plan.nranks)]
        work = dist.all_gather(recv, send, group=group, async_op=True)
        return counts, blocks, recv, work

    def finish(pending):
        counts, blocks, recv, work = pending
        work.wait()
        data = torch.cat([recv[r][:int(counts[r])] for r in range(plan.nranks)], 0)
        return blocks, data

    pending = issue(0) if plan.nbatches else None
    for b in range(plan.nbatches):
        if overlap:
            nxt = issue(b + 1) if b + 1 < plan.nbatches else None
            blocks, data = finish(pending)
        else:
            blocks, data = finish(pending)
            nxt = issue(b + 1) if b + 1 < plan.nbatches else None
        consume(b, blocks, data)
        pending = nxt
    return sent


def allreduce_sum_(tensor, group=None):
    """In-place sum over ranks (steps (iii) and (vii): T3 parts of R1, R2 and W,
    and the local |R3|^2 shares)."""
    import torch.distributed as dist
    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
