"""Replicas on two ranks (gloo, CPU): camera sharding and edit broadcast.

Two processes each hold a copy of the world.  Rank 0 makes crater edits and
broadcasts them; both ranks apply them to their copy and render their shard
of the cameras with the oracle (this host logic needs no GPU).  Rank 0 gathers
the shards and checks them against one process rendering every camera on the
edited world.
"""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _library():
    """The package loads libhf.so on import (no compute call is made here)."""
    import __graft_entry__

    __graft_entry__.build_library()


def test_shard_covers_every_item_once():
    from paper_2608_17390_gb300.replicas import shard

    for n in (0, 1, 5, 64, 101):
        for ws in (1, 2, 3, 8):
            seen = []
            for r in range(ws):
                a, b = shard(n, r, ws)
                seen += list(range(a, b))
                assert b - a in (n // ws, n // ws + 1)
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2608_17390_gb300.replicas import broadcast_edit, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cells, _ = synth.make_grid(96, 80, seed=21, slab_frac=0.3, n_walls=4)
        rng = np.random.default_rng(0)
        for _ in range(3):
            edit = None
            if rank == 0:
                edit = synth.crater_edit(cells, int(rng.integers(0, 96)), int(rng.integers(0, 80)))
            x0, y0, blk = broadcast_edit(edit, src=0)
            cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        cams = synth.c3_cameras(cells, seed=5, n=7, scale=60)
        a, b = shard(len(cams), rank, world)
        mine = [(i, oracle.render(cells, cams[i], shadows=True)) for i in range(a, b)]
        got = [None] * world
        dist.all_gather_object(got, (synth.grid_hash(cells), mine))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


def test_two_replicas_match_one_process():
    import multiprocessing as mp

    import oracle
    import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the same edits in one process
    cells, _ = synth.make_grid(96, 80, seed=21, slab_frac=0.3, n_walls=4)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x0, y0, blk = synth.crater_edit(cells, int(rng.integers(0, 96)), int(rng.integers(0, 80)))
        cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
    assert got[0][0] == got[1][0] == synth.grid_hash(cells)
    cams = synth.c3_cameras(cells, seed=5, n=7, scale=60)
    pieces = sorted(got[0][1] + got[1][1], key=lambda t: t[0])
    assert [i for i, _ in pieces] == list(range(len(cams)))
    for i, res in pieces:
        ref = oracle.render(cells, cams[i], shadows=True)
        for k in ("hit_cell", "layer", "face", "depth", "rgba", "shadow"):
            assert np.array_equal(res[k], ref[k]), (i, k)


def _edit_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import synth
    from paper_2608_17390_gb300 import HFError
    from paper_2608_17390_gb300.replicas import replicated_edit

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cells, _ = synth.make_grid(96, 80, seed=21, slab_frac=0.3, n_walls=4)
        applied = []
        rng = np.random.default_rng(0)
        for _ in range(3):  # rank 0 draws each crater against its own mirror
            edit = None
            if rank == 0:
                edit = synth.crater_edit(cells, int(rng.integers(0, 96)), int(rng.integers(0, 80)))
            replicated_edit(edit, cells, src=0,
                            apply=lambda x0, y0, b: applied.append((x0, y0, b.copy())))
        before = synth.grid_hash(cells)
        errors = []
        bad_slab = np.full((2, 3), synth.pack_cells(10, 20, 15, 1), np.uint32)  # h2 < h1
        for edit in ((5, 6, bad_slab), (95, 0, np.ones((2, 3), np.uint32)),
                     (0, 79, np.ones((2, 1), np.uint32))):
            try:
                replicated_edit(edit if rank == 0 else None, cells, src=0,
                                apply=lambda x0, y0, b: applied.append("applied a bad edit"))
                errors.append(None)
            except HFError as e:
                errors.append(e.code)
        q.put((rank, synth.grid_hash(cells), before,
               [(x0, y0, synth.grid_hash(b)) for x0, y0, b in applied[:3]], len(applied), errors))
    finally:
        dist.destroy_process_group()


def test_replicated_edit_same_on_every_rank_and_bad_edits_refused_everywhere():
    """Rank 0 draws three craters; both ranks apply each one in the same
    order (the stub stands in for hf_edit on a GPU context) and end with the
    same world.  An invalid cell block and rectangles past the grid's edge
    raise the same HFError on both ranks, and neither applies them."""
    import multiprocessing as mp

    import synth
    from paper_2608_17390_gb300 import HF_E_INVALID_ARG, HF_E_OUT_OF_BOUNDS

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_edit_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, h0, b0, a0, n0, e0), (_, h1, b1, a1, n1, e1) = res
    assert h0 == h1 == b0 == b1 and a0 == a1 and n0 == n1 == 3
    assert e0 == e1 == [HF_E_INVALID_ARG, HF_E_OUT_OF_BOUNDS, HF_E_OUT_OF_BOUNDS]
    cells, _ = synth.make_grid(96, 80, seed=21, slab_frac=0.3, n_walls=4)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x0, y0, blk = synth.crater_edit(cells, int(rng.integers(0, 96)), int(rng.integers(0, 80)))
        cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
    assert h0 == synth.grid_hash(cells)
