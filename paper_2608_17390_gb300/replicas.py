"""Running the ray cast on several GPUs: replicas, not partitions.

Every rank holds its own copy of the world (cells + pyramid, at most a few
hundred MiB).  Render work is sharded by camera; the only exchange step is
an edit: its rectangle of new cells is broadcast from the rank that received
it to every rank, and each rank applies it with hf_edit, which repairs its own
pyramid.  There is no reduction, and outputs stay on the rank that rendered
them.  These helpers use torch.distributed with whatever backend the process
group has (nccl on GPUs, gloo on CPUs).
"""

import numpy as np


def shard(n, rank, world_size):
    """Contiguous [start, end) block of n work items for `rank`: sizes differ
    by at most one, and the blocks cover 0..n-1 once, in rank order."""
    if world_size < 1 or not (0 <= rank < world_size):
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world_size)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def broadcast_edit(edit, src=0, device=None):
    """Broadcast an edit (x0, y0, block uint32 [h, w]) from rank `src`.

    Ranks other than src pass edit=None and receive the same tuple.  The
    rectangle header travels as one int64 tensor, the cells as one int32
    tensor (bit-identical to the uint32 words)."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank()
    hdr = torch.zeros(4, dtype=torch.int64, device=device)
    if rank == src:
        x0, y0, blk = edit
        blk = np.ascontiguousarray(blk, dtype=np.uint32)
        hdr[:] = torch.tensor([x0, y0, blk.shape[1], blk.shape[0]], dtype=torch.int64)
    dist.broadcast(hdr, src)
    x0, y0, w, h = (int(v) for v in hdr.cpu())
    cells = torch.empty(h * w, dtype=torch.int32, device=device)
    if rank == src:
        cells.copy_(torch.from_numpy(blk.reshape(-1).view(np.int32)))
    dist.broadcast(cells, src)
    return x0, y0, cells.cpu().numpy().view(np.uint32).reshape(h, w)
