"""Paired-texel worlds (2 bytes per cell, decoded in the kernels) against the
oracle on the oracle's own decoding of the same texels, and against the
4-byte world of the same cells (GPU only)."""

import os

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare, gpu_render, sample_pixels
from oracle import pairs as opairs

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 4


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _pair_world(W, H, seed, f=0.35):
    cells, _ = synth.make_grid(W, H, seed=seed, slab_frac=f)
    cells = synth.pairify(cells & np.uint32(0x07FFFFFF))  # materials 0..7
    return synth.encode_pairs(cells)


def _pyr_equal(hf, ctx, cells, what):
    for k, lv in enumerate(oracle.pyramid(cells), start=1):
        assert (hf.hf_read_pyramid(ctx, k) == lv).all(), "%s level %d" % (what, k)


def test_pair_world_full_frames_equal_the_oracle(hf):
    tex = _pair_world(96, 80, 21)
    cells = opairs.decode(tex)
    cams = synth.camera_array([
        synth.pose_to_camera(48.5, 5.5, 90.0, 0, -35, 70, 64, 40),
        synth.pose_to_camera(20.25, 60.75, float((cells[60, 20] & 0xFF) + 2), 135, 0, 90, 57, 21),
        synth.pose_to_camera(70.0, 30.0, 200.0, 300, -85, 60, 33, 33),
    ])
    ctx = hf.hf_create_pairs(tex)
    try:
        info = hf.hf_info(ctx)
        assert info["cell_format"] == hf.HF_CELLS_PAIR16 and info["cell_bytes"] == 96 * 80 * 2
        assert (hf.hf_read_cells(ctx, 0, 0, 96, 80) == cells).all()
        assert (hf.hf_read_cells(ctx, 3, 7, 11, 5) == cells[7:12, 3:14]).all()
        _pyr_equal(hf, ctx, cells, "pairs build")
        orc = [oracle.render(cells, c, shadows=True, nthreads=NT) for c in cams]
        for mip in (0, 1, 3, 6):
            for flags in (hf.HF_SHADOWS, hf.HF_SHADOWS | hf.HF_PLAIN):
                g = gpu_render(hf, ctx, cams, shadows=True,
                               opts=hf.make_opts(mip_start=mip, flags=flags))
                for i in range(len(cams)):
                    compare(g[i], orc[i], shadows=True, what="pairs cam %d mip %d" % (i, mip))
    finally:
        hf.hf_destroy(ctx)


def test_pair_world_edits_repair_and_read_back(hf):
    rng = np.random.default_rng(8)
    tex = _pair_world(64, 36, 22, 0.5)
    cells = opairs.decode(tex)
    ctx = hf.hf_create_pairs(tex)
    try:
        for e in range(12):
            w = 2 * int(rng.integers(1, 12))
            h = int(rng.integers(1, 12))
            x0 = 2 * int(rng.integers(0, (64 - w) // 2 + 1))
            y0 = int(rng.integers(0, 36 - h + 1))
            blk, _ = synth.make_grid(w, h, seed=100 + e, slab_frac=0.5)
            blk = synth.pairify(blk & np.uint32(0x07FFFFFF))
            hf.hf_edit(ctx, x0, y0, blk)
            cells[y0:y0 + h, x0:x0 + w] = blk
        hf.hf_sync(ctx)
        assert (hf.hf_read_cells(ctx, 0, 0, 64, 36) == cells).all()
        _pyr_equal(hf, ctx, cells, "pairs repair")
        cam = synth.camera_array([synth.pose_to_camera(32.5, 2.5, 70.0, 10, -40, 80, 48, 30)])
        g = gpu_render(hf, ctx, cam, shadows=True, opts=hf.make_opts(flags=hf.HF_SHADOWS))
        compare(g[0], oracle.render(cells, cam[0], shadows=True), shadows=True, what="after edits")
        # edits the pair encoding cannot hold are refused, and change nothing
        bad_slab = np.array([[synth.pack_cells(1, 5, 9, 0), synth.pack_cells(2, 0, 0, 0)]], np.uint32)
        for x0, blk in ((4, bad_slab), (3, cells[0:1, 3:5].copy()), (4, cells[0:1, 4:7].copy()),
                        (4, np.array([[synth.pack_cells(1, 0, 0, 9), 0]], np.uint32))):
            with pytest.raises(hf.HFError):
                hf.hf_edit(ctx, x0, 0, blk)
        assert (hf.hf_read_cells(ctx, 0, 0, 64, 36) == cells).all()
    finally:
        hf.hf_destroy(ctx)


def test_pair_world_equals_the_word_world_bit_for_bit(hf):
    """The same cells as paired texels and as 4-byte words: every output of
    the batched cameras (resolutions / 8) is identical, and so is the march."""
    c3 = synth.config_c3(scale=8)
    cells = synth.pairify(c3["cells"] & np.uint32(0x07FFFFFF))
    tex = synth.encode_pairs(cells)
    cams = c3["cams"]
    a, b = hf.hf_create(cells), hf.hf_create_pairs(tex)
    try:
        for opts in (hf.make_opts(flags=hf.HF_SHADOWS), hf.make_opts(mip_start=3, tile_w=16,
                                                                     tile_h=8, flags=hf.HF_SHADOWS)):
            ga = gpu_render(hf, a, cams, shadows=True, opts=opts)
            gb = gpu_render(hf, b, cams, shadows=True, opts=opts)
            for i in range(len(cams)):
                for k in ga[i]:
                    assert np.array_equal(ga[i][k], gb[i][k]), (i, k)
        import torch

        ma = hf.alloc_outputs(cams[:8], fields=("hit_cell", "layer", "depth"))
        mb = hf.alloc_outputs(cams[:8], fields=("hit_cell", "layer", "depth"))
        hf.hf_render_march(a, cams[:8], ma, hf.make_march_opts(steps=64, bisections=4))
        hf.hf_render_march(b, cams[:8], mb, hf.make_march_opts(steps=64, bisections=4))
        hf.hf_sync(a)
        hf.hf_sync(b)
        torch.cuda.synchronize()
        for x, y in zip(ma, mb):
            for k in x:
                assert torch.equal(x[k], y[k]), k
        # and the oracle agrees on sampled pixels of two cameras
        for i in (0, 40):
            pix = sample_pixels(int(cams[i]["w"]), int(cams[i]["h"]), 300, i)
            sel = {k: v[pix] for k, v in gb[i].items()}
            compare(sel, oracle.render(cells, cams[i], shadows=True, pix=pix, nthreads=NT),
                    shadows=True, what="pairs C3/8 cam %d" % i)
    finally:
        hf.hf_destroy(a)
        hf.hf_destroy(b)


def test_pair_world_full_size_sampled(hf):
    """The 2048 x 16384 fly-through world in paired texels (64 MiB of cells),
    sampled pixels of three 1920 x 1080 frames in the benchmark's launch
    configuration."""
    cells = synth.pairify(synth.config_c4()["cells"] & np.uint32(0x07FFFFFF))
    tex = synth.encode_pairs(cells)
    cams = synth.config_c4_frames(cells, n_frames=1000)[[0, 500, 999]]
    ctx = hf.hf_create_pairs(tex)
    try:
        assert hf.hf_info(ctx)["cell_bytes"] == 64 << 20
        g = gpu_render(hf, ctx, cams, opts=hf.make_opts(tile_w=8, tile_h=16, mip_start=5))
        for i, c in enumerate(cams):
            pix = sample_pixels(int(c["w"]), int(c["h"]), 400, 50 + i)
            sel = {k: v[pix] for k, v in g[i].items()}
            compare(sel, oracle.render(cells, c, pix=pix, nthreads=NT), what="pairs C4 frame %d" % i)
    finally:
        hf.hf_destroy(ctx)
