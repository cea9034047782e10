"""The comparison marcher (the paper's fixed-step method) vs its CPU oracle.

Both are float32 in the same operation order with no fused multiply-add, so
hit cell, layer and depth must agree bit for bit."""

import numpy as np
import pytest

import synth
from oracle import march

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _gpu(hf, ctx, cams, opts):
    import torch

    outs = hf.alloc_outputs(cams, fields=("hit_cell", "layer", "depth"))
    hf.hf_render_march(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    return [{k: (v.cpu().numpy().view(np.uint32) if k == "hit_cell" else v.cpu().numpy())
             for k, v in o.items()} for o in outs]


@pytest.mark.parametrize("steps,far", [(128, 600.0), (16, 200.0), (512, 600.0)])
def test_march_bit_exact(hf, steps, far):
    cfg = synth.config_c3(scale=24)
    cells, cams = cfg["cells"], cfg["cams"][::5]
    ctx = hf.hf_create(cells)
    try:
        got = _gpu(hf, ctx, cams, hf.make_march_opts(steps=steps, far_dist=far))
        for i, c in enumerate(cams):
            ref = march.march_camera(cells, c, steps=steps, far=far)
            for k in ("hit_cell", "layer"):
                bad = np.nonzero(got[i][k] != ref[k])[0]
                assert bad.size == 0, (i, k, bad[:5])
            assert np.array_equal(got[i]["depth"].view(np.uint32), ref["depth"].view(np.uint32)), i
    finally:
        hf.hf_destroy(ctx)


def test_march_rejects_bad_options(hf):
    cfg = synth.config_c1()
    ctx = hf.hf_create(cfg["cells"])
    try:
        outs = hf.alloc_outputs(cfg["cams"], fields=("hit_cell", "depth"))
        with pytest.raises(hf.HFError):
            hf.hf_render_march(ctx, cfg["cams"], outs, hf.make_march_opts(far_dist=-1.0))
        with pytest.raises(hf.HFError):
            hf.hf_render_march(ctx, cfg["cams"], outs, hf.make_march_opts(steps=70000))
    finally:
        hf.hf_destroy(ctx)
