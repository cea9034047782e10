"""Autotuner: every candidate renders identical buffers; the choice is cached."""

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _host(outs):
    return [{k: t.cpu().numpy().copy() for k, t in o.items()} for o in outs]


def test_every_candidate_gives_identical_buffers(hf, tmp_path):
    import torch

    from paper_2608_17390_gb300.autotune import autotune

    cfg = synth.config_c3(scale=8)
    cells, cams = cfg["cells"], cfg["cams"]
    stream = torch.cuda.Stream()
    ctx = hf.hf_create(cells, stream=stream.cuda_stream)
    try:
        outs = hf.alloc_outputs(cams, shadows=True)
        ref = None
        for tw, th in ((8, 4), (4, 8), (32, 1), (16, 8)):
            for mip in (0, 2, 5, 11):
                hf.hf_render(ctx, cams, outs, hf.make_opts(tile_w=tw, tile_h=th, mip_start=mip,
                                                           flags=hf.HF_SHADOWS))
                hf.hf_sync(ctx)
                got = _host(outs)
                if ref is None:
                    ref = got
                    continue
                for i in range(len(cams)):
                    for k in ref[i]:
                        assert np.array_equal(ref[i][k], got[i][k]), (tw, th, mip, i, k)
        # and the common result is the oracle's (two cameras spot-checked in full)
        for i in (0, 41):
            g = {k: (v.view(np.uint32) if k in ("hit_cell", "rgba") else v) for k, v in ref[i].items()}
            compare(g, oracle.render(cells, cams[i], shadows=True, nthreads=8), shadows=True,
                    what="autotune common result cam %d" % i)
        cache = str(tmp_path / "tune.json")
        opts, table = autotune(ctx, cams, outs, stream, shadows=True, reps=1, cache_file=cache,
                               tiles=((8, 4), (8, 8)), mips=(4, 6))
        assert len(table) == 4 and (opts.tile_w, opts.tile_h) in ((8, 4), (8, 8))
        opts2, table2 = autotune(ctx, cams, outs, stream, shadows=True, cache_file=cache)
        assert table2 == [] and (opts2.tile_w, opts2.tile_h, opts2.mip_start) == (
            opts.tile_w, opts.tile_h, opts.mip_start)
        # host outputs are tuned separately, over the wide tiles, and the tuned
        # render into pinned host buffers gives the same result
        host = hf.alloc_outputs(cams, device="pinned", shadows=True)
        hopts, htable = autotune(ctx, cams, host, stream, shadows=True, reps=1, mips=(5,),
                                 host_outputs=True)
        assert len(htable) == 6 and hopts.flags & hf.HF_HOST_OUTPUTS
        hf.hf_render(ctx, cams, host, hopts)
        hf.hf_sync(ctx)
        for i in range(len(cams)):
            for k in ref[i]:
                assert np.array_equal(ref[i][k], host[i][k].numpy()), ("host", i, k)
    finally:
        hf.hf_destroy(ctx)
