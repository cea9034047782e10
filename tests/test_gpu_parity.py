"""CUDA path vs the oracle, through the C ABI (GPU only).

Full frames at sizes the oracle finishes in seconds (several tiles and ragged
tails), sampled pixels at the configurations' full sizes in the launch
configuration the benchmark times, adversarial single rays, edge cases,
pyramid repair vs rebuild, edit visibility, batched vs plain, every mip level
and tile shape, and the step guard.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare, gpu_render, sample_pixels

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


@pytest.fixture(scope="module")
def c1():
    return synth.config_c1()


@pytest.fixture(scope="module")
def c2grid():
    cfg = synth.config_c2(240, 135)
    return cfg


def _ctx(hf, cells):
    return hf.hf_create(cells)


def _oracle_all(cells, cams, shadows=False):
    return [oracle.render(cells, c, shadows=shadows, nthreads=NT) for c in cams]


def _gather(hf, ctx, cams, pix_per_cam, shadows, opts):
    """Render on the GPU, gather sampled pixels on the device, copy those back."""
    import torch

    outs = hf.alloc_outputs(cams, device="cuda", shadows=shadows)
    hf.hf_render(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    res = []
    for o, pix in zip(outs, pix_per_cam):
        idx = torch.from_numpy(pix).cuda()
        d = {}
        for k, t in o.items():
            a = t[idx].cpu().numpy()
            if k in ("hit_cell", "rgba"):
                a = a.view(np.uint32)
            d[k] = a
        res.append(d)
    return res


# ------------------------------------------------------------ full frames

def test_c1_full_frame(hf, c1):
    ctx = _ctx(hf, c1["cells"])
    try:
        g = gpu_render(hf, ctx, c1["cams"])
        o = _oracle_all(c1["cells"], c1["cams"])
        compare(g[0], o[0], what="C1")
        assert (o[0]["face"] != 255).mean() > 0.5
    finally:
        hf.hf_destroy(ctx)


def test_c1_shadows_full_frame(hf, c1):
    ctx = _ctx(hf, c1["cells"])
    try:
        g = gpu_render(hf, ctx, c1["cams"], shadows=True)
        o = _oracle_all(c1["cells"], c1["cams"], shadows=True)
        compare(g[0], o[0], shadows=True, what="C1 shadows")
        assert 0 < o[0]["shadow"].sum() < o[0]["shadow"].size
    finally:
        hf.hf_destroy(ctx)


@pytest.mark.parametrize("mip", [0, 1, 2, 4, 6, 8, 30])
@pytest.mark.parametrize("tile", [(8, 4), (32, 1), (4, 8), (16, 4), (16, 16)])
def test_c1_every_mip_level_and_tile_shape(hf, c1, mip, tile):
    ctx = _ctx(hf, c1["cells"])
    try:
        opts = hf.make_opts(tile_w=tile[0], tile_h=tile[1], mip_start=mip, flags=hf.HF_SHADOWS)
        g = gpu_render(hf, ctx, c1["cams"], shadows=True, opts=opts)
        o = _oracle_all(c1["cells"], c1["cams"], shadows=True)
        compare(g[0], o[0], shadows=True, what="C1 mip %d tile %s" % (mip, tile))
    finally:
        hf.hf_destroy(ctx)


def test_c2_reduced_full_frame(hf, c2grid):
    ctx = _ctx(hf, c2grid["cells"])
    try:
        g = gpu_render(hf, ctx, c2grid["cams"], shadows=True)
        o = _oracle_all(c2grid["cells"], c2grid["cams"], shadows=True)
        compare(g[0], o[0], shadows=True, what="C2 240x135")
    finally:
        hf.hf_destroy(ctx)


def test_c3_reduced_batch_with_shadows(hf):
    cfg = synth.config_c3(scale=16)
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = _ctx(hf, cells)
    try:
        for flags in (hf.HF_SHADOWS, hf.HF_SHADOWS | hf.HF_PLAIN, hf.HF_SHADOWS | hf.HF_NOGRAPH):
            g = gpu_render(hf, ctx, cams, shadows=True, opts=hf.make_opts(flags=flags))
            o = _oracle_all(cells, cams, shadows=True)
            for i in range(len(cams)):
                compare(g[i], o[i], shadows=True, what="C3/16 cam %d flags %d" % (i, flags))
    finally:
        hf.hf_destroy(ctx)


# ---------------------------------------------- full sizes, sampled pixels

def test_c2_full_size_sampled(hf):
    cfg = synth.config_c2()
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = _ctx(hf, cells)
    try:
        pix = [sample_pixels(1920, 1080, 20000, 5)]
        g = _gather(hf, ctx, cams, pix, True, hf.make_opts(flags=hf.HF_SHADOWS))
        o = oracle.render(cells, cams[0], shadows=True, pix=pix[0], nthreads=NT)
        compare(g[0], o, shadows=True, what="C2 full")
    finally:
        hf.hf_destroy(ctx)


def test_c3_full_size_sampled(hf):
    """The benchmark's workload at full size: 64 cameras, one batched launch,
    shadow rays; the library's default tile and mip start, and the tuned
    launch the benchmark times (4 x 32 tiles, mip start 5)."""
    cfg = synth.config_c3()
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = _ctx(hf, cells)
    try:
        pix = [sample_pixels(int(c["w"]), int(c["h"]), 300, 100 + i) for i, c in enumerate(cams)]
        runs = {"default": _gather(hf, ctx, cams, pix, True, hf.make_opts(flags=hf.HF_SHADOWS)),
                "4x32 mip 5": _gather(hf, ctx, cams, pix, True,
                                      hf.make_opts(tile_w=4, tile_h=32, mip_start=5,
                                                   flags=hf.HF_SHADOWS))}
        for i, c in enumerate(cams):
            o = oracle.render(cells, c, shadows=True, pix=pix[i], nthreads=NT)
            for name, g in runs.items():
                compare(g[i], o, shadows=True, what="C3 %s cam %d" % (name, i))
    finally:
        hf.hf_destroy(ctx)


def test_c4_sampled_frames(hf):
    cells = synth.config_c4()["cells"]
    frames = synth.config_c4_frames(cells, 1000)[::100]
    ctx = _ctx(hf, cells)
    try:
        pix = [sample_pixels(1920, 1080, 1500, 200 + i) for i in range(len(frames))]
        runs = {"default": _gather(hf, ctx, frames, pix, False, hf.make_opts()),
                "4x32 mip 9": _gather(hf, ctx, frames, pix, False,
                                      hf.make_opts(tile_w=4, tile_h=32, mip_start=9))}
        for i, c in enumerate(frames):
            o = oracle.render(cells, c, pix=pix[i], nthreads=NT)
            for name, g in runs.items():
                compare(g[i], o, what="C4 %s frame %d" % (name, 100 * i))
    finally:
        hf.hf_destroy(ctx)


# ------------------------------------------------------ adversarial rays

def _rand_grid(rng, W, H, hmax=12):
    h0 = rng.integers(0, hmax, (H, W))
    slab = rng.random((H, W)) < 0.4
    h1 = np.where(slab, h0 + rng.integers(1, 6, (H, W)), 0)
    h2 = np.where(slab, h1 + rng.integers(0, 5, (H, W)), 0)
    return synth.pack_cells(h0, h1, h2, rng.integers(0, 8, (H, W)))


def test_adversarial_single_rays(hf):
    """1 x 1 cameras = arbitrary integer rays on a quarter-cell lattice, so
    exact corners, boundary starts and grazing heights are frequent."""
    S = 65536
    rng = np.random.default_rng(99)
    for gi in range(6):
        W, H = int(rng.integers(3, 80)), int(rng.integers(3, 80))
        cells = _rand_grid(rng, W, H, hmax=20)
        n = 3000
        o = np.stack([rng.integers(0, 4 * W, n) * S // 4, rng.integers(0, 4 * H, n) * S // 4,
                      rng.integers(0, 120, n) * S // 4], 1)
        d = np.stack([rng.integers(-8, 9, n) * S // 8, rng.integers(-8, 9, n) * S // 8,
                      rng.integers(-8, 9, n) * S // 64], 1)
        o[:500] = np.stack([rng.integers(0, W * S, 500), rng.integers(0, H * S, 500),
                            rng.integers(0, 30 * S, 500)], 1)
        d[:500] = rng.integers(-(1 << 20), 1 << 20, (500, 3))
        cams = synth.camera_array([synth.ray_camera(o[k], d[k]) for k in range(n)])
        orc = oracle.trace_rays(cells, o, d, shadows=True)
        ctx = _ctx(hf, cells)
        try:
            for mip in (0, 2, 7):
                for b in range(0, n, 1000):
                    sub = cams[b:b + 1000]
                    g = gpu_render(hf, ctx, sub, shadows=True,
                                   opts=hf.make_opts(mip_start=mip, flags=hf.HF_SHADOWS))
                    merged = {k: np.concatenate([x[k] for x in g]) for k in g[0]}
                    ref = {k: (None if v is None else v[b:b + 1000]) for k, v in orc.items()}
                    compare(merged, ref, shadows=True, what="grid %d mip %d" % (gi, mip))
        finally:
            hf.hf_destroy(ctx)


def test_edge_cases(hf):
    S = 65536
    rng = np.random.default_rng(7)
    cases = []
    # 1 x 1 grid, non-power-of-two grid, 16384-wide and 16384-tall strips, an
    # image of the largest width, height-zero floor
    cases.append((np.array([[synth.pack_cells(3, 5, 9, 2)]], np.uint32),
                  [synth.pose_to_camera(0.5, 0.5, 7.0, 0, -90, 60, 3, 3),
                   synth.pose_to_camera(0.0, 0.0, 4.0, 45, -10, 90, 5, 4)]))
    cases.append((_rand_grid(rng, 37, 29, 30),
                  [synth.pose_to_camera(18.5, 14.5, 40.0, 10, -90, 80, 33, 17),
                   synth.pose_to_camera(0.0, 28.99, 10.0, 135, -5, 90, 31, 9),
                   synth.pose_to_camera(36.99, 0.0, 2.0, 300, 20, 60, 64, 3)]))
    wide = _rand_grid(rng, 16384, 16, 40)
    cases.append((wide, [synth.pose_to_camera(16383.9, 8.0, 30.0, 270, -1, 20, 97, 5),
                         synth.pose_to_camera(0.1, 8.0, 30.0, 90, -1, 20, 97, 5)]))
    tall = _rand_grid(rng, 16, 16384, 40)
    cases.append((tall, [synth.pose_to_camera(8.0, 16383.9, 30.0, 180, -1, 20, 97, 5),
                         synth.pose_to_camera(8.0, 0.1, 30.0, 0, -1, 20, 97, 5)]))
    cases.append((_rand_grid(rng, 37, 29, 30),
                  [synth.pose_to_camera(18.5, 14.5, 40.0, 30, -30, 120, int(hf.HF_MAX_DIM), 2)]))
    cases.append((np.zeros((8, 8), np.uint32),
                  [synth.pose_to_camera(4.0, 4.0, 3.0, 0, -90, 90, 7, 7)]))
    for cells, poses in cases:
        cams = synth.camera_array(poses)
        ctx = _ctx(hf, cells)
        try:
            g = gpu_render(hf, ctx, cams, shadows=True,
                           opts=hf.make_opts(flags=hf.HF_SHADOWS))
            for i, c in enumerate(cams):
                o = oracle.render(cells, c, shadows=True)
                compare(g[i], o, shadows=True, what="edge %s cam %d" % (cells.shape, i))
            # an empty batch is a no-op
            hf.hf_render(ctx, cams[:0], [])
        finally:
            hf.hf_destroy(ctx)


def test_camera_heights_at_node_tops_and_in_caves(hf):
    """Cameras exactly at a pyramid node's top height, one 2^-16 unit above
    it, inside a slab cave, on an exact cell corner, and on the grid's corner
    looking out (origins outside the grid are rejected by validation):
    the level a camera's rays start from depends on these comparisons, and
    every start must give the oracle's image at every mip."""
    rng = np.random.default_rng(2024)
    cells = _rand_grid(rng, 96, 80, hmax=40)
    levels = oracle.pyramid(cells)  # levels 1..L, byte 2 = max top
    poses = []
    for k, (x, y) in enumerate([(40.0, 33.0), (10.5, 70.25), (77.0, 12.0)]):
        cx, cy = int(x), int(y)
        h0, h1, h2, _ = synth.unpack_cells(cells[cy, cx])
        top0 = int(h2) if int(h1) > int(h0) else int(h0)
        tops = [top0] + [int((lv[cy >> (i + 1), cx >> (i + 1)] >> 16) & 0xFF)
                         for i, lv in enumerate(levels)]
        for lvl in (0, 2, 4):
            for dz in (0.0, 1.0 / 65536):
                poses.append(synth.pose_to_camera(x, y, tops[lvl] + dz, 97.0 * k + 31 * lvl,
                                                  -20.0 + 10 * lvl, 80, 23, 11))
    cave = np.argwhere((synth.unpack_cells(cells)[1] > synth.unpack_cells(cells)[0] + 1))[0]
    h0, h1, _, _ = synth.unpack_cells(cells[cave[0], cave[1]])
    poses.append(synth.pose_to_camera(cave[1] + 0.5, cave[0] + 0.5, (int(h0) + int(h1)) / 2.0,
                                      200, 5, 90, 31, 9))
    poses.append(synth.pose_to_camera(0.0, 0.0, 50.0, 225, -30, 70, 27, 13))
    poses.append(synth.pose_to_camera(48.0, 40.0, 45.0, 225, -45, 70, 27, 13))
    cams = synth.camera_array(poses)
    ctx = _ctx(hf, cells)
    try:
        orc = [oracle.render(cells, c, shadows=True) for c in cams]
        for mip in (0, 1, 3, 5, 7):
            g = gpu_render(hf, ctx, cams, shadows=True,
                           opts=hf.make_opts(mip_start=mip, flags=hf.HF_SHADOWS))
            for i in range(len(cams)):
                compare(g[i], orc[i], shadows=True, what="cam %d mip %d" % (i, mip))
    finally:
        hf.hf_destroy(ctx)


def test_vertical_rays_hit_height_zero(hf):
    """Odd image sizes put a pixel exactly on the optical axis: with pitch -90
    that ray is vertical; height zero must be hit from above (the paper's
    evaluation section records the z >= 0 guard that made it unhittable)."""
    cells = np.zeros((16, 16), np.uint32)
    cam = synth.camera_array([synth.pose_to_camera(8.0, 8.0, 5.0, 0, -90, 60, 9, 9)])
    ctx = _ctx(hf, cells)
    try:
        g = gpu_render(hf, ctx, cam)
        assert (g[0]["face"] == 5).all()
        assert g[0]["depth"][40] == pytest.approx(5.0, rel=1e-6)
        compare(g[0], oracle.render(cells, cam[0]), what="vertical")
    finally:
        hf.hf_destroy(ctx)


# ------------------------------------------------------- pyramid and edits

def _pyr_equal(hf, ctx, cells, what):
    ref = oracle.pyramid(cells)
    for k, lv in enumerate(ref, start=1):
        got = hf.hf_read_pyramid(ctx, k)
        assert got.shape == lv.shape and (got == lv).all(), "%s level %d" % (what, k)


def _extreme_cells(rng, W, H):
    """Valid cells at the ends of every byte range: no slab at h0 = 0 and 255,
    slabs [h0+1, 255], [255, 255], [1, 1] over h0 = 0, materials 0 and 255."""
    kinds = [(0, 0, 0), (255, 0, 0), (254, 255, 255), (0, 1, 1), (0, 255, 255), (7, 8, 200),
             (100, 0, 0)]
    k = rng.integers(0, len(kinds), (H, W))
    h0 = np.array([t[0] for t in kinds])[k]
    h1 = np.array([t[1] for t in kinds])[k]
    h2 = np.array([t[2] for t in kinds])[k]
    mat = rng.choice([0, 1, 128, 255], (H, W))
    return synth.pack_cells(h0, h1, h2, mat)


def test_cells_read_back_unchanged_at_byte_extremes(hf):
    """The device keeps its own cell layout; what goes in through hf_create and
    hf_edit comes back unchanged through hf_read_cells, and the pyramid and
    renders see the same cells as the oracle."""
    rng = np.random.default_rng(255)
    W, H = 77, 45
    cells = _extreme_cells(rng, W, H)
    assert hf.hf_validate_cells(cells)[0] == hf.HF_OK
    ctx = _ctx(hf, cells)
    try:
        assert (hf.hf_read_cells(ctx, 0, 0, W, H) == cells).all()
        blk = _extreme_cells(rng, 20, 9)
        hf.hf_edit(ctx, 50, 30, blk)
        cells[30:39, 50:70] = blk
        hf.hf_sync(ctx)
        assert (hf.hf_read_cells(ctx, 0, 0, W, H) == cells).all()
        assert (hf.hf_read_cells(ctx, 49, 29, 13, 7) == cells[29:36, 49:62]).all()
        _pyr_equal(hf, ctx, cells, "extremes")
        cams = synth.camera_array([synth.pose_to_camera(38.5, 22.5, 300.0, 30, -70, 80, 41, 23),
                                   synth.pose_to_camera(10.5, 5.5, 120.0, 60, -10, 90, 41, 23)])
        g = gpu_render(hf, ctx, cams, shadows=True, opts=hf.make_opts(flags=hf.HF_SHADOWS))
        for i, c in enumerate(cams):
            compare(g[i], oracle.render(cells, c, shadows=True), shadows=True,
                    what="extremes cam %d" % i)
    finally:
        hf.hf_destroy(ctx)


def test_pyramid_build_and_repair_equal_rebuild(hf):
    rng = np.random.default_rng(3)
    for W, H in ((300, 200), (64, 64), (1, 70), (129, 3)):
        cells = _rand_grid(rng, W, H, 200)
        ctx = _ctx(hf, cells)
        try:
            _pyr_equal(hf, ctx, cells, "build %dx%d" % (W, H))
            for e in range(25):
                w = int(rng.integers(1, min(W, 70) + 1))
                h = int(rng.integers(1, min(H, 70) + 1))
                if e == 0:
                    w, h = W, H
                x0 = int(rng.integers(0, W - w + 1))
                y0 = int(rng.integers(0, H - h + 1))
                blk = _rand_grid(rng, w, h, 240)
                hf.hf_edit(ctx, x0, y0, blk)
                cells[y0:y0 + h, x0:x0 + w] = blk
            hf.hf_sync(ctx)
            assert (hf.hf_read_cells(ctx, 0, 0, W, H) == cells).all()
            _pyr_equal(hf, ctx, cells, "repair %dx%d" % (W, H))
            hf.hf_rebuild(ctx)
            _pyr_equal(hf, ctx, cells, "rebuild %dx%d" % (W, H))
        finally:
            hf.hf_destroy(ctx)


def test_edit_visible_next_render_and_equals_fresh_world(hf, c1):
    cells = c1["cells"].copy()
    cams = c1["cams"]
    ctx = _ctx(hf, cells)
    try:
        import torch

        before = hf.alloc_outputs(cams, shadows=True)
        hf.hf_render(ctx, cams, before, hf.make_opts(flags=hf.HF_SHADOWS))  # issued before
        for cx, cy in ((128, 60), (100, 90), (3, 250)):
            x0, y0, blk = synth.crater_edit(cells, cx, cy)
            hf.hf_edit(ctx, x0, y0, blk)
            cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        after = gpu_render(hf, ctx, cams, shadows=True)
        torch.cuda.synchronize()
        b = {k: v.cpu().numpy() for k, v in before[0].items()}
        compare({k: (v.view(np.uint32) if k in ("hit_cell", "rgba") else v) for k, v in b.items()},
                oracle.render(c1["cells"], cams[0], shadows=True), shadows=True,
                what="render issued before the edit")
        fresh = _ctx(hf, cells)
        try:
            f = gpu_render(hf, fresh, cams, shadows=True)
        finally:
            hf.hf_destroy(fresh)
        for k in f[0]:
            assert (f[0][k] == after[0][k]).all(), k
        compare(after[0], oracle.render(cells, cams[0], shadows=True), shadows=True,
                what="after edit")
        assert (after[0]["hit_cell"] != b["hit_cell"].view(np.uint32)).any()
    finally:
        hf.hf_destroy(ctx)


def test_renders_on_other_streams_respect_edit_order(hf, c1):
    import torch

    cells = c1["cells"].copy()
    cams = c1["cams"]
    ctx = _ctx(hf, cells)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        a = hf.alloc_outputs(cams)
        hf.hf_render(ctx, cams, a, hf.make_opts(stream=s1.cuda_stream))
        x0, y0, blk = synth.crater_edit(cells, 128, 60)
        hf.hf_edit(ctx, x0, y0, blk)
        cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        b = hf.alloc_outputs(cams)
        hf.hf_render(ctx, cams, b, hf.make_opts(stream=s2.cuda_stream))
        hf.hf_sync(ctx)
        torch.cuda.synchronize()
        ga = {k: v.cpu().numpy() for k, v in a[0].items()}
        gb = {k: v.cpu().numpy() for k, v in b[0].items()}
        fix = lambda d: {k: (v.view(np.uint32) if k in ("hit_cell", "rgba") else v) for k, v in d.items()}
        compare(fix(ga), oracle.render(c1["cells"], cams[0]), what="stream 1 before edit")
        compare(fix(gb), oracle.render(cells, cams[0]), what="stream 2 after edit")
    finally:
        hf.hf_destroy(ctx)


# ------------------------------------------------------------ guard, stats

def test_step_guard_reports_and_context_survives(hf, c1):
    ctx = _ctx(hf, c1["cells"])
    try:
        outs = hf.alloc_outputs(c1["cams"])
        with pytest.raises(hf.HFError) as e:
            hf.hf_render(ctx, c1["cams"], outs,
                         hf.make_opts(max_steps=3, mip_start=0, flags=hf.HF_SYNC))
        assert e.value.code == hf.HF_E_STEP_LIMIT
        face = outs[0]["face"].cpu().numpy()
        assert (face == hf.HF_FACE_ERROR).any()
        assert hf.hf_sync(ctx) is None  # flag cleared
        g = gpu_render(hf, ctx, c1["cams"])
        compare(g[0], oracle.render(c1["cells"], c1["cams"][0]), what="after guard")
    finally:
        hf.hf_destroy(ctx)


def test_invalid_render_arguments(hf, c1):
    ctx = _ctx(hf, c1["cells"])
    try:
        outs = hf.alloc_outputs(c1["cams"])
        for tw, th in ((3, 8), (2, 2), (512, 1)):
            with pytest.raises(hf.HFError) as e:
                hf.hf_render(ctx, c1["cams"], outs, hf.make_opts(tile_w=tw, tile_h=th))
            assert e.value.code == hf.HF_E_INVALID_ARG
        bad = c1["cams"].copy()
        bad[0]["o"][0] = 256 * 65536
        with pytest.raises(hf.HFError) as e:
            hf.hf_render(ctx, bad, outs)
        assert e.value.code == hf.HF_E_INVALID_ARG
        with pytest.raises(hf.HFError) as e:
            hf.hf_edit(ctx, 250, 250, np.zeros((10, 10), np.uint32))
        assert e.value.code == hf.HF_E_OUT_OF_BOUNDS
    finally:
        hf.hf_destroy(ctx)


def test_flat_fetch_counter_matches_oracle_steps(hf, c1):
    """With mip_start 0 the kernel reads exactly one cell per visited cell:
    its counter must equal the oracle's count of visited cells (every C1 ray
    descends, so the oracle's above-the-terrain exit never applies)."""
    ctx = _ctx(hf, c1["cells"])
    try:
        outs = hf.alloc_outputs(c1["cams"])
        hf.hf_stats(ctx)
        hf.hf_render(ctx, c1["cams"], outs, hf.make_opts(mip_start=0, flags=hf.HF_STATS))
        st = hf.hf_stats(ctx)
        o = oracle.render(c1["cells"], c1["cams"][0], nthreads=NT)
        assert st["rays"] == 320 * 240
        assert st["node_fetches"] == 0
        assert st["cell_fetches"] == int(o["steps"].sum())
    finally:
        hf.hf_destroy(ctx)


def test_nowait_admission_reports_busy(hf):
    """Admission without waiting: when every render slot is in flight,
    HF_NOWAIT returns HF_E_BUSY instead of blocking; nothing is lost."""
    cfg = synth.config_c3(scale=2)
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = _ctx(hf, cells)
    try:
        info = hf.hf_info(ctx)
        outs = hf.alloc_outputs(cams)
        busy = 0
        for _ in range(info["render_slots"] + 4):
            try:
                hf.hf_render(ctx, cams, outs, hf.make_opts(flags=hf.HF_NOWAIT))
            except hf.HFError as e:
                assert e.code == hf.HF_E_BUSY
                busy += 1
        hf.hf_sync(ctx)
        assert busy >= 1
        g = gpu_render(hf, ctx, cams[:2])
        for i in range(2):
            pix = sample_pixels(int(cams[i]["w"]), int(cams[i]["h"]), 300, i)
            o = oracle.render(cells, cams[i], pix=pix, nthreads=NT)
            compare({k: v[pix] for k, v in g[i].items()}, o, what="after busy cam %d" % i)
    finally:
        hf.hf_destroy(ctx)


def test_host_outputs_equal_device_outputs(hf, c1):
    """HF_HOST_OUTPUTS: the kernel writes pinned host buffers itself; the
    results equal the device-buffer render bit for bit, and pageable host
    memory is rejected before anything runs."""
    import torch

    cells, cams = c1["cells"], c1["cams"]
    ctx = _ctx(hf, cells)
    try:
        dev = gpu_render(hf, ctx, cams, shadows=True, opts=hf.make_opts(flags=hf.HF_SHADOWS))
        for extra in (0, hf.HF_NOGRAPH):
            host = hf.alloc_outputs(cams, device="pinned", shadows=True)
            hf.hf_render(ctx, cams, host,
                         hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_HOST_OUTPUTS | hf.HF_SYNC | extra))
            for k, t in host[0].items():
                assert (t.numpy() == dev[0][k].view(t.numpy().dtype)).all(), k
        pageable = [{k: torch.empty(v.shape, dtype=v.dtype) for k, v in o.items()} for o in host]
        with pytest.raises(hf.HFError):
            hf.hf_render(ctx, cams, pageable,
                         hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_HOST_OUTPUTS))
        hf.hf_sync(ctx)
    finally:
        hf.hf_destroy(ctx)


def test_host_staged_outputs_equal_device_outputs(hf, c1):
    """HF_HOST_STAGED: the library renders chunks into its own staging and
    copies each back while the next renders; the host buffers equal a device
    render bit for bit, for one camera and for a multi-chunk batch with some
    fields absent, with each field's buffers back to back (one copy per run)
    and apart; pageable memory and conflicting flags are refused."""
    import torch

    for cells, cams, fields, sh in (
            (c1["cells"], c1["cams"], ("hit_cell", "layer", "face", "depth", "rgba", "shadow"), True),
            (synth.config_c3(scale=8)["cells"], synth.config_c3(scale=8)["cams"],
             ("hit_cell", "depth", "rgba"), False),
            # with shadow rays and every field
            (synth.config_c3(scale=8)["cells"], synth.config_c3(scale=8)["cams"],
             ("hit_cell", "layer", "face", "depth", "rgba", "shadow"), True)):
        ctx = _ctx(hf, cells)
        try:
            flags = hf.HF_SHADOWS if sh else 0
            dev = gpu_render(hf, ctx, cams, shadows=sh, opts=hf.make_opts(flags=flags), fields=fields)
            for rep in range(3):  # later calls reuse the staging buffers
                host = hf.alloc_outputs(cams, device="pinned", shadows=sh, fields=fields)
                if rep == 2:  # one allocation per camera and field: no two buffers adjacent
                    host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                             for k, v in o.items()} for o in host]
                hf.hf_render(ctx, cams, host, hf.make_opts(flags=flags | hf.HF_HOST_STAGED | hf.HF_SYNC))
                for i in range(len(cams)):
                    for k, t in host[i].items():
                        assert (t.numpy() == dev[i][k].view(t.numpy().dtype)).all(), (rep, i, k)
            pageable = [{k: torch.empty(v.shape, dtype=v.dtype) for k, v in o.items()} for o in host]
            with pytest.raises(hf.HFError):
                hf.hf_render(ctx, cams, pageable, hf.make_opts(flags=flags | hf.HF_HOST_STAGED))
            for bad in (hf.HF_HOST_OUTPUTS, hf.HF_PLAIN, hf.HF_NOWAIT):
                with pytest.raises(hf.HFError):
                    hf.hf_render(ctx, cams, host, hf.make_opts(flags=flags | hf.HF_HOST_STAGED | bad))
            hf.hf_sync(ctx)
        finally:
            hf.hf_destroy(ctx)


def _window(cam, x0, y0, w, h):
    """Pixels [x0, x0 + w) x [y0, y0 + h) of a camera, as a camera of their own
    (the same rays: fwd moved to the window's centre)."""
    o, f, r, u, w0, h0 = cam
    a, b = 2 * x0 + w - w0, h0 - h - 2 * y0
    return (o, tuple(f[i] + a * r[i] + b * u[i] for i in range(3)), r, u, w, h)


def test_host_staged_row_bands_equal_the_oracle(hf, c1):
    """HF_HOST_STAGED renders chunks of equal pixel counts (here about ten),
    splitting cameras into row bands: a batch of cameras one pixel wide or
    high, of odd sizes, and two far larger than a chunk equals the oracle
    pixel for pixel."""
    cells = c1["cells"]
    base = synth.pose_to_camera(60.5, 80.25, 120.0, 30.0, -30.0, 70.0, 2560, 1600)
    wins = [(0, 0, 1, 1), (5, 3, 1, 37), (100, 200, 45, 1), (7, 9, 33, 17), (0, 0, 2560, 1600),
            (300, 10, 7, 200), (1600, 1200, 2, 2), (100, 50, 1000, 777)]
    cams = synth.camera_array([_window(base, *wn) for wn in wins])
    ctx = _ctx(hf, cells)
    try:
        for rep in range(2):
            host = hf.alloc_outputs(cams, device="pinned", shadows=True)
            hf.hf_render(ctx, cams, host,
                         hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_HOST_STAGED | hf.HF_SYNC))
            for i, c in enumerate(cams):
                g = {k: t.numpy().view(np.uint32) if k in ("hit_cell", "rgba") else t.numpy()
                     for k, t in host[i].items()}
                compare(g, oracle.render(cells, c, shadows=True, nthreads=NT), shadows=True,
                        what="rep %d window %s" % (rep, wins[i]))
    finally:
        hf.hf_destroy(ctx)
