"""Full-frame parity at the configurations' full sizes (GPU only).

Every pixel of every image is compared with the oracle (hit cell, layer, face
and shadow bit exact; depth within 1e-5 relative; colour within 1/255), in the
launch configuration the benchmark times and in the library's default one:

* the eye-level 1920 x 1080 view over the 2048 x 2048 world with walls and
  caves, with shadow rays;
* all 64 cameras of the batched-cameras workload (16 x 3840 x 2160,
  24 x 1920 x 1080, 24 x 640 x 360, 188,006,400 primary rays plus shadow
  rays), one batched launch, tuned (4 x 32 tiles, mip start 5), default and
  plain (one launch per camera), the three bit-identical;
* every 100th frame of the 1000-frame fly-through over the 2048 x 16384
  world, tuned (4 x 32, mip start 9) and default;
* the serving loop on the 2048 x 16384 world at the serving resolutions
  (640 x 360 to 3840 x 2160) with crater edits every 11th request: each served
  image equals the same request rendered alone on a fresh world holding
  exactly the edits before it, bit for bit, and the oracle on that world
  (every pixel up to 1920 x 1080, 40,000 sampled pixels per 3840 x 2160 image);
* the largest grid, 16384 x 16384 (1 GiB of cells), with rays that cross all
  of it and a camera at the highest allowed altitude, and its pyramid and
  shadow bounds after large edits against a fresh build;
* the largest batch (4096 cameras) and the largest image (16384 x 16384).

The paper evaluates its renderers against a CPU ray cast (Section 4.1); here
the CPU ray cast is the oracle and the bar is exact.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare, sample_pixels

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


def _host(out, pix=None):
    """One camera's device outputs as numpy arrays (optionally at pix)."""
    import torch

    d = {}
    idx = None if pix is None else torch.from_numpy(np.asarray(pix, np.int64)).cuda()
    for k, t in out.items():
        a = (t if idx is None else t[idx]).cpu().numpy()
        if k in ("hit_cell", "rgba"):
            a = a.view(np.uint32)
        d[k] = a
    return d


def _render(hf, ctx, cams, shadows, opts):
    import torch

    outs = hf.alloc_outputs(cams, device="cuda", shadows=shadows)
    hf.hf_render(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    return outs


def _assert_identical(a, b, what):
    import torch

    for k in a:
        assert torch.equal(a[k], b[k]), "%s: %s differs" % (what, k)


def test_c2_full_frame_at_1080p(hf):
    cfg = synth.config_c2()
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = hf.hf_create(cells)
    try:
        g = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS))
        b = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_NOGRAPH,
                                                      tile_w=4, tile_h=32))
        _assert_identical(g[0], b[0], "C2 default vs 4x32")
        o = oracle.render(cells, cams[0], shadows=True, nthreads=NT)
        compare(_host(g[0]), o, shadows=True, what="C2 1920x1080")
        assert (o["face"] != 255).mean() > 0.3 and 0 < o["shadow"].sum()
    finally:
        hf.hf_destroy(ctx)


def test_c3_every_camera_full_frame(hf):
    """The benchmark's batched workload, every pixel of every camera."""
    cfg = synth.config_c3()
    cells, cams = cfg["cells"], cfg["cams"]
    assert sum(int(c["w"]) * int(c["h"]) for c in cams) == 188006400
    ctx = hf.hf_create(cells)
    try:
        tuned = _render(hf, ctx, cams, True,
                        hf.make_opts(tile_w=4, tile_h=32, mip_start=5, flags=hf.HF_SHADOWS))
        default = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS))
        plain = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_PLAIN))
        for i in range(len(cams)):
            _assert_identical(tuned[i], default[i], "C3 cam %d tuned vs default" % i)
            _assert_identical(tuned[i], plain[i], "C3 cam %d batched vs plain" % i)
        del default, plain
        hits = 0
        for i, c in enumerate(cams):
            o = oracle.render(cells, c, shadows=True, nthreads=NT)
            compare(_host(tuned[i]), o, shadows=True, what="C3 cam %d (%dx%d)" % (
                i, int(c["w"]), int(c["h"])))
            hits += int((o["face"] != 255).sum())
        assert hits > 0.5 * 188006400
    finally:
        hf.hf_destroy(ctx)


def test_c4_every_100th_frame_full(hf):
    cells = synth.config_c4()["cells"]
    frames = synth.config_c4_frames(cells, 1000)[::100]
    ctx = hf.hf_create(cells)
    try:
        tuned = _render(hf, ctx, frames, False, hf.make_opts(tile_w=4, tile_h=32, mip_start=9))
        default = _render(hf, ctx, frames, False, hf.make_opts())
        for i in range(len(frames)):
            _assert_identical(tuned[i], default[i], "C4 frame %d tuned vs default" % (100 * i))
        del default
        for i, c in enumerate(frames):
            o = oracle.render(cells, c, nthreads=NT)
            compare(_host(tuned[i]), o, what="C4 frame %d" % (100 * i))
    finally:
        hf.hf_destroy(ctx)


def test_c5_serving_on_the_large_world(hf):
    """The native serving loop on the 2048 x 16384 world at the serving
    resolutions, edits interleaved 10 renders : 1 crater, several batches in
    flight on separate lanes."""
    import torch

    cells = synth.config_c4()["cells"]
    records = synth.poisson_requests(cells, 44, rate=4000.0, seed=21, edit_every=11)
    renders = [i for i, r in enumerate(records) if r["kind"] == "render"]
    assert len(renders) == 40 and {(int(records[i]["cam"]["w"]), int(records[i]["cam"]["h"]))
                                   for i in renders} == set(synth.SERVING_RESOLUTIONS)
    outs = [None if r["kind"] == "edit" else hf.alloc_outputs(np.array([r["cam"]]))[0]
            for r in records]
    ctx = hf.hf_create(cells)
    try:
        res = hf.hf_serve_replay(ctx, records, lanes=8, max_batch=8, output_budget=4 << 30,
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
        if j > k:  # renders k..j-1 were admitted after the same edits
            fresh = hf.hf_create(world)
            try:
                for i in range(k, j):
                    cam = np.array([records[i]["cam"]])
                    assert int(res["version"][i]) == sum(
                        r["kind"] == "edit" for r in records[:i])
                    alone = _render(hf, fresh, cam, False, hf.make_opts())
                    _assert_identical(outs[i], alone[0], "served request %d vs alone" % i)
                    w, h = int(cam[0]["w"]), int(cam[0]["h"])
                    pix = None if w * h <= 1920 * 1080 else sample_pixels(w, h, 40000, i)
                    o = oracle.render(world, cam[0], pix=pix, nthreads=NT)
                    compare(_host(outs[i], pix), o, what="served request %d (%dx%d)" % (i, w, h))
                    checked += 1
            finally:
                hf.hf_destroy(fresh)
        if j < len(records):  # the edit at j
            x0, y0, blk = records[j]["edit"]
            world[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        k = j + 1
    assert checked == 40


def _max_world(seed=11):
    """A 16384 x 16384 world (the largest grid, 1 GiB of cells): 64-cell
    blocks of random height with per-cell noise, a few 200-high ridges, and
    slabs over about a tenth of the cells."""
    n = int(16384)
    rng = np.random.default_rng(seed)
    h0 = np.repeat(np.repeat(rng.integers(0, 120, (n // 64, n // 64), dtype=np.uint8), 64, 0), 64, 1)
    h0 += rng.integers(0, 8, (n, n), dtype=np.uint8)
    h0[4096::4096, :] = 200
    h0[:, 6000] = 200
    slab = (rng.integers(0, 10, (n, n), dtype=np.uint8) == 0) & (h0 < 200)
    h1 = np.where(slab, h0 + 10, 0).astype(np.uint8)
    h2 = np.where(slab, h1 + 6, 0).astype(np.uint8)
    return synth.pack_cells(h0, h1, h2, h0 & 7)


def test_largest_grid_and_camera_extremes(hf):
    """The largest grid (16384 x 16384) with shadow rays: rays that cross the
    whole world and leave it at the far corner, a camera at the highest
    allowed altitude (z just under 2^28 fixed-point units) looking straight
    down over 14,000 cells, and one in the far corner looking back; every
    pixel equals the oracle, and the batched and plain launches agree."""
    cells = _max_world()
    cams = synth.camera_array([
        synth.pose_to_camera(0.5, 0.5, 150.0, 45, -0.06, 20, 48, 12),
        synth.pose_to_camera(8192.5, 8192.5, 4095.0, 0, -90, 120, 64, 64),
        synth.pose_to_camera(16383.5, 16383.5, 140.0, 225, 0.5, 90, 33, 9)])
    ctx = hf.hf_create(cells)
    try:
        opts = hf.make_opts(flags=hf.HF_SHADOWS)
        g = _render(hf, ctx, cams, True, opts)
        p = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_PLAIN))
        for i in range(len(cams)):
            _assert_identical(g[i], p[i], "camera %d batched vs plain" % i)
        for i, c in enumerate(cams):
            compare(_host(g[i]), oracle.render(cells, c, shadows=True, nthreads=NT), shadows=True,
                    what="largest grid, camera %d" % i)
    finally:
        hf.hf_destroy(ctx)


def test_largest_batch_and_largest_image(hf):
    """The batch limit and the image limit, with shadow rays: HF_MAX_CAMERAS
    (4096) small cameras in one batched launch equal the plain launches and
    the oracle, one camera more is refused; a 16384 x 16384 image (268 M
    primary rays) is identical from the plain and the batched kernel and
    equals the oracle on 100,000 sampled pixels."""
    import torch

    cells = synth.config_c1()["cells"]
    rng = np.random.default_rng(3)
    n = int(hf.HF_MAX_CAMERAS)
    poses = [synth.pose_to_camera(float(rng.uniform(1, 255)), float(rng.uniform(1, 255)),
                                  float(rng.uniform(20, 250)), float(rng.uniform(0, 360)),
                                  float(rng.uniform(-89, 10)), float(rng.uniform(40, 100)), 8, 4)
             for _ in range(n + 1)]
    cams = synth.camera_array(poses)
    ctx = hf.hf_create(cells)
    try:
        with pytest.raises(hf.HFError) as e:
            hf.hf_render(ctx, cams, hf.alloc_outputs(cams, shadows=True),
                         hf.make_opts(flags=hf.HF_SHADOWS))
        assert e.value.code == hf.HF_E_INVALID_ARG
        cams = cams[:n]
        g = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS))
        p = _render(hf, ctx, cams, True, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_PLAIN))
        for i in range(n):
            _assert_identical(g[i], p[i], "camera %d of the largest batch" % i)
        for i in range(0, n, 97):
            compare(_host(g[i]), oracle.render(cells, cams[i], shadows=True), shadows=True,
                    what="largest batch, camera %d" % i)

        big = synth.camera_array([synth.pose_to_camera(128.5, 128.5, 200.0, 30, -60, 100,
                                                       16384, 16384)])
        a = _render(hf, ctx, big, True, hf.make_opts(flags=hf.HF_SHADOWS))
        b = _render(hf, ctx, big, True, hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_NOGRAPH))
        _assert_identical(a[0], b[0], "largest image, plain vs batched")
        del b
        pix = sample_pixels(16384, 16384, 100000, 17)
        compare(_host(a[0], pix), oracle.render(cells, big[0], shadows=True, pix=pix, nthreads=NT),
                shadows=True, what="largest image")
        del a
        torch.cuda.empty_cache()
    finally:
        hf.hf_destroy(ctx)


def test_largest_grid_edits_repair_pyramid_and_bounds(hf):
    """Edits on the largest grid after a shadowed render: a full-width strip
    across the 2^27-cell index (rows 8180-8219) and a crater in the far
    corner.  The repaired pyramid levels and shadow bounds equal a fresh
    world's bit for bit, and the renders equal the oracle on the edited cells."""
    cells = _max_world(seed=12)
    cams = synth.camera_array([
        synth.pose_to_camera(8192.5, 8150.5, 300.0, 0, -20, 90, 64, 32),
        synth.pose_to_camera(16300.5, 16250.5, 120.0, 30, -30, 90, 48, 24)])
    rng = np.random.default_rng(13)
    strip = synth.pack_cells(rng.integers(0, 150, (40, 16384)), 0, 0, rng.integers(0, 8, (40, 16384)))
    ctx = hf.hf_create(cells)
    fresh = None
    try:
        opts = hf.make_opts(flags=hf.HF_SHADOWS)
        _render(hf, ctx, cams, True, opts)  # builds the shadow bounds
        hf.hf_edit(ctx, 0, 8180, strip)
        cells[8180:8220, :] = strip
        x0, y0, blk = synth.crater_edit(cells, 16330, 16340)
        hf.hf_edit(ctx, x0, y0, blk)
        cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        g = _render(hf, ctx, cams, True, opts)
        hf.hf_sync(ctx)
        fresh = hf.hf_create(cells)
        _render(hf, fresh, cams, True, opts)
        hf.hf_sync(fresh)
        for level in (1, 2, 5, 9, 14):
            assert np.array_equal(hf.hf_read_pyramid(ctx, level), hf.hf_read_pyramid(fresh, level)), \
                "pyramid level %d after edits differs from a fresh build" % level
        got, s1 = hf.hf_read_sun_bounds(ctx)
        want, s2 = hf.hf_read_sun_bounds(fresh)
        assert s1 == s2 and np.array_equal(got, want), "repaired shadow bounds differ from a fresh build"
        for i, c in enumerate(cams):
            compare(_host(g[i]), oracle.render(cells, c, shadows=True, nthreads=NT), shadows=True,
                    what="largest grid after edits, camera %d" % i)
    finally:
        hf.hf_destroy(ctx)
        if fresh is not None:
            hf.hf_destroy(fresh)
