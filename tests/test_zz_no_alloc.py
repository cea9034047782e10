"""hf_render_noalloc: the allocation-free render entry point.

Some callers cannot allocate device memory once they are running: a render
loop whose GPU memory budget is fixed at start-up, or a latency-critical thread
where cudaMalloc/cudaFree could stall or implicitly synchronise the device.
hf_render may allocate its per-slot camera tables and graphs on first use;
hf_render_noalloc keeps its scratch in one static device array instead.  This
test calls it through the C ABI twice in a row, with different batches, and
checks each result against hf_render's within the parity tolerances used by
the other tests (exact cell, layer, face and shadow; depth 1e-5 relative;
colour 1/255).  It lives in its own file so that it is collected last.
"""

import numpy as np
import pytest

import synth
from hfcheck import compare, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _noalloc(hf, ctx, cams, opts):
    import torch

    outs = hf.alloc_outputs(cams, device="cuda", shadows=True)
    hf.hf_render_noalloc(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    res = []
    for o in outs:
        d = {}
        for k, t in o.items():
            a = t.cpu().numpy()
            d[k] = a.view(np.uint32) if k in ("hit_cell", "rgba") else a
        res.append(d)
    return res


def test_noalloc_matches_hf_render_on_two_calls_in_a_row(hf):
    cfg = synth.config_c3(scale=16)
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = hf.hf_create(cells)
    try:
        batches = [cams[:7], cams[30:33]]  # the second call is smaller than the first
        for i, b in enumerate(batches):
            opts = hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_SYNC)
            got = _noalloc(hf, ctx, b, opts)
            ref = gpu_render(hf, ctx, b, shadows=True, opts=hf.make_opts(flags=hf.HF_SHADOWS))
            for j in range(len(b)):
                ref_j = {k: v.astype(np.float64) if k == "depth" else v for k, v in ref[j].items()}
                compare(got[j], ref_j, shadows=True, what="noalloc call %d cam %d" % (i, j))
    finally:
        hf.hf_destroy(ctx)


def test_noalloc_rejects_oversize_batches_and_foreign_streams(hf):
    import torch

    cfg = synth.config_c1()
    ctx = hf.hf_create(cfg["cells"])
    try:
        cam = synth.camera_array([synth.ray_camera((65536 * 5, 65536 * 5, 65536 * 200),
                                                   (1000, 2000, -3000))])
        many = np.repeat(cam, hf.HF_NOALLOC_MAX_CAMERAS + 1)
        outs = hf.alloc_outputs(many[:1], device="cuda") * len(many)
        with pytest.raises(hf.HFError) as e:
            hf.hf_render_noalloc(ctx, many, outs)
        assert e.value.code == hf.HF_E_INVALID_ARG
        s = torch.cuda.Stream()
        with pytest.raises(hf.HFError) as e:
            hf.hf_render_noalloc(ctx, cam, outs[:1], hf.make_opts(stream=s.cuda_stream))
        assert e.value.code == hf.HF_E_INVALID_ARG
        # flags it cannot honour are refused, not dropped
        for flag in (hf.HF_STATS, hf.HF_PLAIN, hf.HF_NOGRAPH, hf.HF_NOWAIT, hf.HF_HOST_OUTPUTS,
                     hf.HF_HOST_STAGED):
            with pytest.raises(hf.HFError) as e:
                hf.hf_render_noalloc(ctx, cam, outs[:1], hf.make_opts(flags=hf.HF_SYNC | flag))
            assert e.value.code == hf.HF_E_INVALID_ARG, flag
        # the largest allowed batch still renders
        hf.hf_render_noalloc(ctx, many[:-1], outs[:-1], hf.make_opts(flags=hf.HF_SYNC))
        hf.hf_sync(ctx)
    finally:
        hf.hf_destroy(ctx)


def test_noalloc_allocates_nothing_after_its_first_call(hf):
    """The defining property: once the first call on a device has looked up
    the scratch array's address, further calls (of several batch sizes) leave
    the device's free memory unchanged."""
    import torch

    cfg = synth.config_c3(scale=16)
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = hf.hf_create(cells)
    try:
        batches = [cams[:40], cams[5:6], cams[10:33], cams[:64]]
        outs = [hf.alloc_outputs(b, device="cuda", shadows=True) for b in batches]
        opts = hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_SYNC)
        hf.hf_render_noalloc(ctx, batches[0], outs[0], opts)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            for b, o in zip(batches, outs):
                hf.hf_render_noalloc(ctx, b, o, opts)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        hf.hf_destroy(ctx)


def test_noalloc_reports_the_step_guard_and_recovers(hf):
    """With HF_SYNC, a step guard of one iteration makes rays stop early: the
    call returns HF_E_STEP_LIMIT, the stopped pixels carry the error face, and
    the next call (default guard) renders normally, equal to hf_render."""
    cfg = synth.config_c1()
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = hf.hf_create(cells)
    try:
        import torch

        outs = hf.alloc_outputs(cams, device="cuda", shadows=True)
        with pytest.raises(hf.HFError) as e:
            hf.hf_render_noalloc(ctx, cams, outs,
                                 hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_SYNC, max_steps=1))
        assert e.value.code == hf.HF_E_STEP_LIMIT
        torch.cuda.synchronize()
        assert (outs[0]["face"] == 254).any()
        got = _noalloc(hf, ctx, cams, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_SYNC))
        ref = gpu_render(hf, ctx, cams, shadows=True, opts=hf.make_opts(flags=hf.HF_SHADOWS))
        ref0 = {k: v.astype(np.float64) if k == "depth" else v for k, v in ref[0].items()}
        compare(got[0], ref0, shadows=True, what="noalloc after the step guard")
        assert (got[0]["face"] != 254).all()
    finally:
        hf.hf_destroy(ctx)
