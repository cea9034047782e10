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


def replicated_edit(edit, cells, src=0, device=None, apply=None):
    """One edit of the replicated world: the exchange step of the multi-GPU
    path.

    Rank `src` passes edit = (x0, y0, block) and the others None.  The edit is
    broadcast (broadcast_edit); then every rank checks it the way hf_edit does
    on the host before any device work -- the rectangle inside its grid
    (HF_E_OUT_OF_BOUNDS) and every cell a valid two-interval word
    (hf_validate_cells, HF_E_INVALID_ARG) -- so that a bad edit raises the same
    HFError on every rank and no replica applies it.  A valid edit is passed to
    `apply(x0, y0, block)` (hf_edit on the rank's context; None for host-only
    use) and written into the rank's host mirror `cells`.  Returns the edit."""
    from . import HF_E_OUT_OF_BOUNDS, HF_OK, HFError, hf_validate_cells

    x0, y0, blk = broadcast_edit(edit, src=src, device=device)
    H, W = cells.shape
    h, w = blk.shape
    if w == 0 or h == 0 or x0 < 0 or y0 < 0 or x0 + w > W or y0 + h > H:
        raise HFError(HF_E_OUT_OF_BOUNDS, "replicated_edit")
    rc, _ = hf_validate_cells(blk)
    if rc != HF_OK:
        raise HFError(rc, "replicated_edit")
    if apply is not None:
        apply(x0, y0, blk)
    cells[y0:y0 + h, x0:x0 + w] = blk
    return x0, y0, blk
