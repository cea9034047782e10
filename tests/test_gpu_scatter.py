"""The scattered renderer (the paper's Scattered method) against its oracle,
through the C ABI (GPU only): the packed screen bit for bit, the resolved
outputs, batches, paired-texel worlds, edits and argument checks."""

import os

import numpy as np
import pytest

import synth
from oracle import pairs as opairs
from oracle import scatter as oscatter

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


def _run(hf, ctx, cams, fps, nu, nv, nz, depth_max, raw=False):
    import torch

    outs = hf.alloc_outputs(cams, fields=("hit_cell", "layer", "face", "depth", "rgba"))
    flags = hf.HF_SYNC | (hf.HF_SCATTER_RAW if raw else 0)
    hf.hf_render_scatter(ctx, cams, outs, fps,
                         hf.make_scatter_opts(nu=nu, nv=nv, nz=nz, depth_max=depth_max, flags=flags))
    torch.cuda.synchronize()
    res = []
    for o in outs:
        d = {k: t.cpu().numpy() for k, t in o.items()}
        d["hit_cell"] = d["hit_cell"].view(np.uint32)
        d["rgba"] = d["rgba"].view(np.uint32)
        res.append(d)
    return res


def _check(got, want, what):
    for k in ("hit_cell", "layer", "face"):
        bad = np.nonzero(got[k] != want[k])[0]
        assert bad.size == 0, "%s %s at %d pixels, first %s" % (what, k, bad.size, bad[:5])
    assert np.array_equal(got["depth"].view(np.uint32), want["depth"].view(np.uint32)), what + " depth"
    g = got["rgba"].view(np.uint8).reshape(-1, 4).astype(int)
    o = want["rgba"].view(np.uint8).reshape(-1, 4).astype(int)
    assert np.abs(g - o).max(initial=0) <= 1, what + " rgba"


CASES = [(256, 256, 8, 512.0), (1024, 1024, 16, 1024.0), (300, 777, 5, 333.0)]


@pytest.mark.parametrize("nu,nv,nz,dmax", CASES)
def test_packed_screen_and_resolve_equal_the_oracle(hf, nu, nv, nz, dmax):
    cfg = synth.config_c1()
    cells = cfg["cells"]
    cams = synth.camera_array([tuple(cfg["cams"][0][k] for k in ("o", "f", "r", "u", "w", "h")),
                               synth.pose_to_camera(30.5, 200.0, 60.0, 150.0, -60.0, 75, 97, 61),
                               synth.pose_to_camera(128.0, 128.0, 200.0, 10.0, -90.0, 60, 64, 64),
                               synth.pose_to_camera(20.0, 20.0, 250.0, 45.0, 30.0, 60, 33, 17)])
    fps = synth.footprints(cams)
    ctx = hf.hf_create(cells)
    try:
        raw = _run(hf, ctx, cams, fps, nu, nv, nz, dmax, raw=True)
        res = _run(hf, ctx, cams, fps, nu, nv, nz, dmax)
        for i, cam in enumerate(cams):
            args = (nu, nv, nz, *[float(v) for v in fps[i]], dmax)
            want = oscatter.render(cells, cam, *args)
            bad = np.nonzero(raw[i]["hit_cell"] != want["packed"])[0]
            assert bad.size == 0, "cam %d packed screen differs at %d pixels" % (i, bad.size)
            _check(res[i], want, "cam %d" % i)
        # the camera looking up at the sky scatters nothing
        assert (raw[3]["hit_cell"] == 0xFFFFFFFF).all() and (res[3]["layer"] == 255).all()
        # one camera at a time gives the batch's result
        one = _run(hf, ctx, cams[1:2], fps[1:2], nu, nv, nz, dmax)
        for k in one[0]:
            assert np.array_equal(one[0][k], res[1][k]), k
    finally:
        hf.hf_destroy(ctx)


def test_paired_world_and_edits(hf):
    cells, _ = synth.make_grid(200, 160, seed=31, slab_frac=0.4)
    cells = synth.pairify(cells & np.uint32(0x07FFFFFF))
    tex = synth.encode_pairs(cells)
    cams = synth.camera_array([synth.pose_to_camera(100.0, 5.0, 90.0, 0.0, -30.0, 80, 80, 50),
                               synth.pose_to_camera(20.0, 80.0, 70.0, 90.0, -10.0, 90, 64, 36)])
    fps = synth.footprints(cams)
    ctx = hf.hf_create_pairs(tex)
    try:
        for step in range(2):
            res = _run(hf, ctx, cams, fps, 512, 512, 12, 700.0)
            for i, cam in enumerate(cams):
                want = oscatter.render(opairs.decode(tex), cam, 512, 512, 12,
                                       *[float(v) for v in fps[i]], 700.0)
                _check(res[i], want, "pairs step %d cam %d" % (step, i))
            # an edit is seen by the next scatter render
            blk = synth.pairify(synth.make_grid(40, 30, seed=77, slab_frac=0.8)[0] & np.uint32(0x07FFFFFF))
            hf.hf_edit(ctx, 80, 40, blk)
            cells[40:70, 80:120] = blk
            tex = synth.encode_pairs(cells)
    finally:
        hf.hf_destroy(ctx)


def test_scatter_arguments_are_checked(hf):
    cfg = synth.config_c1()
    cams = cfg["cams"]
    ctx = hf.hf_create(cfg["cells"])
    try:
        no_screen = hf.alloc_outputs(cams, fields=("depth",))
        with pytest.raises(hf.HFError):
            hf.hf_render_scatter(ctx, cams, no_screen)
        outs = hf.alloc_outputs(cams)
        for opts in (hf.make_scatter_opts(nz=1), hf.make_scatter_opts(nu=9000),
                     hf.make_scatter_opts(depth_max=-1.0)):
            with pytest.raises(hf.HFError):
                hf.hf_render_scatter(ctx, cams, outs, None, opts)
        with pytest.raises(hf.HFError):
            hf.hf_render_scatter(ctx, cams, outs, np.array([[5.0, 5.0, 1.0, 1.0]], np.float32))
        # defaults (library footprint, 1024 x 1024 x 16) run
        hf.hf_render_scatter(ctx, cams, outs, None, hf.make_scatter_opts(flags=hf.HF_SYNC))
    finally:
        hf.hf_destroy(ctx)
