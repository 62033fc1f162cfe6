"""Edge-row transport of a search sharded by midpoint slabs (tt_search_slab).

A long line is cut into contiguous slabs of CMPs, one per GPU (one process
per GPU, ranks in slab order). At every exchange generation a slab sends the
bests of its first m0 row to the previous rank and of its last row to the
next rank, and receives theirs into its own memory; nothing else crosses
slabs. This module only moves those rows with torch.distributed point-to-
point operations (NCCL between GPUs, gloo on the host); the search itself
runs in the library.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def halo_exchange(rank: int, world: int, group=None):
    """An ``exchange`` for tt_search_slab on rank ``rank`` of ``world``
    slabs: sends send_first to rank - 1 and send_last to rank + 1, receives
    recv_prev from rank - 1 and recv_next from rank + 1, and waits for the
    transfers (with NCCL the wait orders the current stream after them)."""

    def exchange(gen, send_first, send_last, recv_prev, recv_next):
        ops = []
        if rank > 0:
            ops.append(dist.P2POp(dist.isend, send_first, rank - 1, group))
            ops.append(dist.P2POp(dist.irecv, recv_prev, rank - 1, group))
        if rank < world - 1:
            ops.append(dist.P2POp(dist.isend, send_last, rank + 1, group))
            ops.append(dist.P2POp(dist.irecv, recv_next, rank + 1, group))
        if ops:
            for work in dist.batch_isend_irecv(ops):
                work.wait()

    return exchange


__all__ = ["halo_exchange"]
