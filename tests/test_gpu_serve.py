"""Serving loop: each result is the same alone and in the mix.

Requests of mixed sizes are served with edits interleaved, several batches in
flight on separate lanes at once.  Every served render is then re-rendered
alone, on a fresh world holding exactly the edits made before the request was
admitted, and must match bit for bit; two are also checked against the oracle.
"""

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare, sample_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def test_each_result_same_alone_and_in_the_mix(hf):
    import torch

    from paper_2608_17390_gb300 import serve

    cells, _ = synth.make_grid(512, 512, seed=11, slab_frac=0.3, n_walls=20)
    reqs = serve.requests_from(synth.poisson_requests(
        cells, 60, rate=2e4, seed=3, edit_every=7,
        resolutions=((160, 90), (320, 180), (96, 64), (640, 360))))
    srv = serve.Server(cells, lanes=4, max_batch=3, mem_bytes=64 << 20)
    try:
        done = srv.run(reqs, keep_outputs=True)
    finally:
        srv.close()
    renders = [r for r in done if r.kind == "render"]
    edits = sorted([r for r in done if r.kind == "edit"], key=lambda r: r.version)
    assert len(renders) + len(edits) == 60 and len(edits) == 8
    assert srv.batches > 3 and srv.max_inflight >= 2, (srv.batches, srv.max_inflight)
    versions = {r.version for r in renders}
    assert len(versions) > 2
    stats = serve.summarize(done, 1.0)
    assert stats["frame_ms_p50"] is not None and stats["edit_to_visible_ms_p50"] is not None
    # replay: world after the first v edits, each request rendered alone
    world = cells.copy()
    applied = 0
    checked = 0
    for v in sorted(versions):
        while applied < v:
            x0, y0, blk = edits[applied].edit
            world[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
            applied += 1
        ctx = hf.hf_create(world)
        try:
            for r in [r for r in renders if r.version == v]:
                cam = np.array([r.cam])
                alone = hf.alloc_outputs(cam)
                hf.hf_render(ctx, cam, alone, hf.make_opts(flags=hf.HF_SYNC))
                torch.cuda.synchronize()
                for k in alone[0]:
                    a = alone[0][k].cpu().numpy()
                    m = r.outs[k].cpu().numpy()
                    assert np.array_equal(a, m), (r.rid, k, v)
                checked += 1
                if checked in (1, 17):
                    pix = sample_pixels(int(r.cam["w"]), int(r.cam["h"]), 200, r.rid)
                    g = {k: (t.cpu().numpy()[pix].view(np.uint32) if k in ("hit_cell", "rgba")
                             else t.cpu().numpy()[pix]) for k, t in r.outs.items()}
                    compare(g, oracle.render(world, r.cam, pix=pix, nthreads=8),
                            what="served request %d" % r.rid)
        finally:
            hf.hf_destroy(ctx)
    assert checked == len(renders)


def test_native_loop_orders_edits_and_leaves_the_edited_world(hf):
    """hf_serve_replay: every render's version is the number of edits before it
    in the stream, edits are numbered in order, times are sane, and the world
    afterwards holds exactly the edited cells."""
    from paper_2608_17390_gb300 import serve

    cells, _ = synth.make_grid(512, 512, seed=13, slab_frac=0.3, n_walls=20)
    records = synth.poisson_requests(cells, 120, rate=2e4, seed=5, edit_every=6,
                                     resolutions=((160, 90), (320, 180), (96, 64), (640, 360)))
    ctx = hf.hf_create(cells)
    try:
        done = serve.run_native(ctx, records, lanes=4, max_batch=3, mem_bytes=64 << 20)
        edits_before = 0
        world = cells.copy()
        for rec, r in zip(records, done):
            if rec["kind"] == "edit":
                edits_before += 1
                assert r.version == edits_before
                # done is the device completion of the edit, on the host clock
                assert r.admitted >= r.arrival - 1e-4 and r.done >= r.admitted - 1e-4
                x0, y0, blk = rec["edit"]
                world[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
            else:
                assert r.version == edits_before
                assert r.admitted >= r.arrival - 1e-4 and r.done >= r.admitted - 1e-3
        assert edits_before == sum(rec["kind"] == "edit" for rec in records) > 5
        assert len({r.batch_id for r in done if r.kind == "render"}) > 3
        stats = serve.summarize(done, 1.0)
        assert stats["renders"] + stats["edits"] == 120 and stats["frame_ms_p99"] is not None
        got = hf.hf_read_cells(ctx, 0, 0, 512, 512)
        assert np.array_equal(got, world)
    finally:
        hf.hf_destroy(ctx)


def test_native_loop_arguments_are_checked(hf):
    cells, _ = synth.make_grid(64, 64, seed=2, slab_frac=0.3)
    records = synth.poisson_requests(cells, 12, rate=1e4, seed=1, edit_every=5,
                                     resolutions=((64, 48),))
    ctx = hf.hf_create(cells)
    try:
        for kw in (dict(lanes=0), dict(lanes=65), dict(max_batch=0), dict(output_budget=0),
                   dict(flags=hf.HF_PLAIN), dict(output_budget=1000)):
            with pytest.raises(hf.HFError):
                hf.hf_serve_replay(ctx, records, **kw)
        late = [dict(r) for r in records]
        late[3]["arrival"], late[4]["arrival"] = late[4]["arrival"] + 1.0, late[3]["arrival"]
        with pytest.raises(hf.HFError):
            hf.hf_serve_replay(ctx, late)
        assert hf.hf_serve_replay(ctx, []).size == 0
        res = hf.hf_serve_replay(ctx, records, lanes=2, max_batch=2, output_budget=1 << 20)
        assert (res["done"] > 0).all()
    finally:
        hf.hf_destroy(ctx)


def test_native_loop_results_same_alone_and_in_the_mix(hf):
    """Renders served by hf_serve_replay into the caller's buffers equal, bit
    for bit, each request rendered alone on a fresh world holding exactly the
    edits that came before it in the stream."""
    import torch

    cells, _ = synth.make_grid(512, 512, seed=17, slab_frac=0.3, n_walls=20)
    records = synth.poisson_requests(cells, 60, rate=2e4, seed=9, edit_every=7,
                                     resolutions=((160, 90), (320, 180), (96, 64), (640, 360)))
    outs = [None if r["kind"] == "edit" else hf.alloc_outputs(np.array([r["cam"]]))[0]
            for r in records]
    ctx = hf.hf_create(cells)
    try:
        res = hf.hf_serve_replay(ctx, records, lanes=4, max_batch=3, output_budget=64 << 20,
                                 outputs=outs)
        hf.hf_sync(ctx)
        torch.cuda.synchronize()
    finally:
        hf.hf_destroy(ctx)
    assert len(set(res["batch"][res["batch"] != 0xFFFFFFFF])) > 3
    world = cells.copy()
    checked = 0
    k = 0
    while k < len(records):
        j = k
        while j < len(records) and records[j]["kind"] == "render":
            j += 1
        if j > k:  # renders k..j-1 see the same world
            cams = np.array([records[i]["cam"] for i in range(k, j)])
            fresh = hf.hf_create(world)
            try:
                alone = [hf.alloc_outputs(cams[q:q + 1])[0] for q in range(len(cams))]
                for q in range(len(cams)):
                    hf.hf_render(fresh, cams[q:q + 1], [alone[q]])
                hf.hf_sync(fresh)
                torch.cuda.synchronize()
                for q, i in enumerate(range(k, j)):
                    for f, t in outs[i].items():
                        assert torch.equal(t, alone[q][f]), (i, f)
                    checked += 1
            finally:
                hf.hf_destroy(fresh)
        if j < len(records):  # the edit at j
            x0, y0, blk = records[j]["edit"]
            world[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        k = j + 1
    assert checked == sum(r["kind"] == "render" for r in records)
