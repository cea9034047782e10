"""RayVoxel (the paper's voxel-accelerated march) against its oracle through
the C ABI (GPU only): the occupancy pyramid word for word after a build and
after edits, and the traversal's hits bit for bit."""

import os

import numpy as np
import pytest

import oracle
import synth
from oracle import pairs as opairs
from oracle import voxel as ovox

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


def _levels_for(nx0, ny0, nz0):
    levels = 1
    while levels < 16 and max(nx0, ny0, nz0) > (8 << (levels - 1)):
        levels += 1
    return levels


def _check_words(hf, ctx, cells, v, levels, what):
    for l, lv in enumerate(ovox.pyramid(cells, *v, levels)):
        got = hf.hf_read_voxels(ctx, l)
        want = ovox.pack(lv)
        assert got.shape == want.shape and np.array_equal(got, want), "%s level %d" % (what, l)


def _rand_grid(rng, W, H, hmax=150):
    h0 = rng.integers(0, hmax, (H, W))
    slab = rng.random((H, W)) < 0.4
    h1 = np.where(slab, np.minimum(255, h0 + rng.integers(1, 60, (H, W))), 0)
    h2 = np.where(slab, np.minimum(255, h1 + rng.integers(0, 40, (H, W))), 0)
    return synth.pack_cells(h0, h1, h2, rng.integers(0, 8, (H, W)))


@pytest.mark.parametrize("v", [(4, 8, 2), (1, 1, 1), (3, 5, 7), (8, 8, 16)])
def test_build_and_repair_equal_the_oracle(hf, v):
    rng = np.random.default_rng(sum(v))
    W, H = 70, 53
    cells = _rand_grid(rng, W, H)
    ctx = hf.hf_create(cells)
    try:
        levels = _levels_for(-(-W // v[0]), -(-H // v[1]), -(-256 // v[2]))
        hf.hf_voxel_build(ctx, *v)
        _check_words(hf, ctx, cells, v, levels, "build")
        for e in range(8):
            w, h = int(rng.integers(1, 25)), int(rng.integers(1, 20))
            x0, y0 = int(rng.integers(0, W - w + 1)), int(rng.integers(0, H - h + 1))
            blk = _rand_grid(rng, w, h, hmax=250)
            hf.hf_edit(ctx, x0, y0, blk)
            cells[y0:y0 + h, x0:x0 + w] = blk
        hf.hf_sync(ctx)
        _check_words(hf, ctx, cells, v, levels, "repair")
        hf.hf_rebuild(ctx)
        _check_words(hf, ctx, cells, v, levels, "rebuild")
    finally:
        hf.hf_destroy(ctx)


def _render(hf, ctx, cams, opts):
    import torch

    outs = hf.alloc_outputs(cams, fields=("hit_cell", "layer", "depth"))
    hf.hf_render_voxel(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    return [{k: t.cpu().numpy() for k, t in o.items()} for o in outs]


def _compare(got, want, what):
    assert np.array_equal(got["hit_cell"].view(np.uint32), want["hit_cell"]), what + " hit_cell"
    assert np.array_equal(got["layer"], want["layer"]), what + " layer"
    assert np.array_equal(got["depth"].view(np.uint32), want["depth"].view(np.uint32)), what + " depth"


def _cams(W, H, cells):
    return synth.camera_array([
        synth.pose_to_camera(W / 2, 3.0, 150.0, 0.0, -35.0, 70, 48, 30),
        synth.pose_to_camera(10.5, H / 2, float((cells[H // 2, 10] & 0xFF) + 3), 80.0, -2.0, 90, 40, 20),
        synth.pose_to_camera(W / 2, H / 2, 300.0, 30.0, -90.0, 60, 32, 32),
        synth.pose_to_camera(W - 5.0, H - 5.0, 90.0, 225.0, 10.0, 60, 24, 16),
        synth.pose_to_camera(W / 3, H / 3, 400.0, 100.0, -20.0, 80, 36, 20),
    ])


@pytest.mark.parametrize("v,levels,inner,outer", [((4, 8, 2), 0, 4, 1024), ((2, 2, 2), 0, 3, 1024),
                                                  ((5, 3, 4), 1, 2, 4096), ((4, 4, 4), 0, 4, 9)])
def test_traversal_equals_the_oracle(hf, v, levels, inner, outer):
    rng = np.random.default_rng(7)
    W, H = 96, 80
    cells = _rand_grid(rng, W, H)
    cams = _cams(W, H, cells)
    ctx = hf.hf_create(cells)
    try:
        hf.hf_voxel_build(ctx, *v, levels)
        L = levels or _levels_for(-(-W // v[0]), -(-H // v[1]), -(-256 // v[2]))
        g = ovox.Grid(cells, *v, L)
        got = _render(hf, ctx, cams, hf.make_voxel_opts(outer=outer, inner=inner, far_dist=600.0))
        for i, cam in enumerate(cams):
            want = ovox.trace(g, cam["o"], oracle.ray_dirs(cam), far=600.0, outer=outer, inner=inner)
            _compare(got[i], want, "v %s cam %d" % (v, i))
    finally:
        hf.hf_destroy(ctx)


def test_paired_world_and_edits_keep_the_traversal_exact(hf):
    cells, _ = synth.make_grid(128, 96, seed=12, slab_frac=0.4)
    cells = synth.pairify(cells & np.uint32(0x07FFFFFF))
    ctx = hf.hf_create_pairs(synth.encode_pairs(cells))
    cams = _cams(128, 96, cells)
    try:
        hf.hf_voxel_build(ctx, 4, 8, 2)
        L = _levels_for(32, 12, 128)
        blk = synth.pairify(synth.make_grid(30, 20, seed=3, slab_frac=0.9)[0] & np.uint32(0x07FFFFFF))
        hf.hf_edit(ctx, 40, 30, blk)
        cells[30:50, 40:70] = blk
        _check_words(hf, ctx, cells, (4, 8, 2), L, "pairs")
        got = _render(hf, ctx, cams, None)
        g = ovox.Grid(cells, 4, 8, 2, L)
        for i, cam in enumerate(cams):
            _compare(got[i], ovox.trace(g, cam["o"], oracle.ray_dirs(cam)), "pairs cam %d" % i)
    finally:
        hf.hf_destroy(ctx)


def test_voxel_arguments_are_checked(hf):
    cfg = synth.config_c1()
    ctx = hf.hf_create(cfg["cells"])
    try:
        outs = hf.alloc_outputs(cfg["cams"], fields=("hit_cell", "layer", "depth"))
        with pytest.raises(hf.HFError):
            hf.hf_render_voxel(ctx, cfg["cams"], outs)  # no pyramid yet
        for bad in ((0, 8, 2), (65, 8, 2), (4, 8, 300)):
            with pytest.raises(hf.HFError):
                hf.hf_voxel_build(ctx, *bad)
        with pytest.raises(hf.HFError):
            hf.hf_voxel_build(ctx, 4, 8, 2, 17)
        hf.hf_voxel_build(ctx, 4, 8, 2)
        with pytest.raises(hf.HFError):
            hf.hf_render_voxel(ctx, cfg["cams"], outs, hf.make_voxel_opts(far_dist=-1.0))
        hf.hf_render_voxel(ctx, cfg["cams"], outs, hf.make_voxel_opts(flags=hf.HF_SYNC))
    finally:
        hf.hf_destroy(ctx)


def test_full_size_world_sampled(hf):
    """The 2048 x 16384 world with the paper's publication grid (4, 8, 2):
    18.29 MiB of occupancy; sampled pixels of the protocol views."""
    cells = synth.config_c4()["cells"]
    cams = synth.protocol_cameras(cells)[[0, 4, 8, 11]]
    ctx = hf.hf_create(cells)
    try:
        hf.hf_voxel_build(ctx, 4, 8, 2)
        L = _levels_for(512, 2048, 128)
        words = sum(hf.hf_read_voxels(ctx, l).size for l in range(L))
        assert abs(words * 4 / 2**20 - 18.29) < 0.01, words * 4 / 2**20
        got = _render(hf, ctx, cams, None)
        g = ovox.Grid(cells, 4, 8, 2, L)
        from hfcheck import sample_pixels

        for i, cam in enumerate(cams):
            pix = sample_pixels(int(cam["w"]), int(cam["h"]), 500, 90 + i)
            want = ovox.trace(g, cam["o"], oracle.ray_dirs(cam)[pix])
            _compare({k: v[pix] for k, v in got[i].items()}, want, "full cam %d" % i)
    finally:
        hf.hf_destroy(ctx)
