"""Per-cell shadow bounds (hf_sun.cu) against the oracle (GPU only).

The bounds let a shadow ray skip its traversal when its origin lies at or
below F (occluded) or at or above G (lit) of its start cell.  Checked here:

* soundness, straight against the oracle: for every cell of small worlds,
  shadow rays from the cell's extreme and middle positions (the half-open
  extents the start-cell rule gives) at exactly height F and G are traced by
  the oracle, which must find them occluded and lit;
* shadowed renders equal the oracle for suns along every octant, along an
  axis, exactly diagonal, steep, near and at the lowest sun that has bounds
  (a reach of 1024 columns), and for suns without bounds (below the horizon,
  vertical, too low, and one column of reach too low);
* incremental repair after edits equals a fresh build bit for bit, and a
  render after edits equals the oracle on the edited world;
* a change of sun rebuilds the bounds (renders alternate between two suns);
* shadowed renders on two streams around an edit see the old and the new
  world, and the native serving loop with shadow rays (lanes in flight,
  craters in between) gives every request the oracle's image of its world.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from hfcheck import compare, gpu_render

pytestmark = pytest.mark.gpu
S = 65536
NT = os.cpu_count() or 4

SUNS = [
    (321060, -321060, 262144),    # the default: exactly diagonal, 30 deg
    (300000, 120000, 200000),     # x-major, +x +y
    (-300000, 120000, 250000),    # x-major, -x +y
    (-110000, -380000, 300000),   # y-major, -x -y
    (90000, 400000, 150000),      # y-major, +x +y
    (400000, 0, 300000),          # along +x
    (0, -400000, 300000),         # along -y
    (-250000, -250000, 400000),   # diagonal, steep
    (400000, 100000, 100000),     # low: close to the lowest sun with bounds
    (401000, 37000, 100000),      # the lowest: floor(255 * 4.01) + 2 = 1024 columns of reach
]
NO_BOUNDS = [
    (300000, 100000, -50000),     # below the horizon
    (0, 0, 400000),               # vertical
    (400000, 0, 20000),           # too low: rays need > 1024 cells to clear 255
    (401400, 37000, 100000),      # just too low: floor(255 * 4.014) + 2 = 1025 columns
]


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _world(seed, W, H):
    cells, _ = synth.make_grid(W, H, seed=seed, slab_frac=0.35, n_walls=max(1, W // 12))
    return cells


def _bounds(hf, ctx, sun):
    """Build the bounds of `sun` with one shadowed render and read them back."""
    cam = synth.camera_array([synth.ray_camera((S * 2 + 5, S * 2 + 7, S * 250), (1000, 1300, -9000))])
    hf.hf_render(ctx, cam, hf.alloc_outputs(cam, shadows=True),
                 hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_SYNC, sun=sun))
    fg, s = hf.hf_read_sun_bounds(ctx)
    assert s == tuple(sun)
    return fg


def _extent(c, d):
    """Fixed-point end points and middle of cell c's half-open extent along an
    axis for a ray with direction component d (the start-cell rule)."""
    lo, hi = c * S, (c + 1) * S
    if d < 0:
        return (lo + 1, hi, lo + S // 2 + 1)
    return (lo, hi - 1, lo + S // 2)


@pytest.mark.parametrize("sun", SUNS)
def test_bounds_sound_against_the_oracle(hf, sun):
    W, H = 40, 34
    cells = _world(3 + abs(sun[0]) % 7, W, H)
    ctx = hf.hf_create(cells)
    try:
        fg = _bounds(hf, ctx, sun)
    finally:
        hf.hf_destroy(ctx)
    F = (fg & 0xFFFF).astype(np.int64) << 8
    G = (fg >> 16).astype(np.int64) << 8
    o, want = [], []
    for y in range(H):
        ys = _extent(y, sun[1])
        for x in range(W):
            xs = _extent(x, sun[0])
            for px in xs:
                for py in ys:
                    o.append((px, py, F[y, x]))
                    want.append(1)
                    o.append((px, py, G[y, x]))
                    want.append(0)
    o = np.array(o, np.int64)
    d = np.tile(np.array(sun, np.int64), (len(o), 1))
    r = oracle.trace_rays(cells, o, d)
    occluded = (r["face"] != 255).astype(int)
    bad = np.nonzero(occluded != np.array(want))[0]
    assert bad.size == 0, [(tuple(o[k]), want[k]) for k in bad[:5]]
    # the bounds decide something: most cells have F at or above their floor
    h0 = (cells & 0xFF).astype(np.int64) * S
    assert (F >= h0).all() and (G > F).all()


@pytest.mark.parametrize("sun", SUNS + NO_BOUNDS)
def test_shadowed_renders_equal_the_oracle_for_every_sun(hf, sun):
    cfg = synth.config_c3(scale=32)
    cells, cams = cfg["cells"], cfg["cams"][::4]
    ctx = hf.hf_create(cells)
    try:
        opts = hf.make_opts(flags=hf.HF_SHADOWS, sun=sun)
        g = gpu_render(hf, ctx, cams, shadows=True, opts=opts)
        if sun in NO_BOUNDS:
            with pytest.raises(hf.HFError):
                hf.hf_read_sun_bounds(ctx)
    finally:
        hf.hf_destroy(ctx)
    for i, c in enumerate(cams):
        o = oracle.render(cells, c, shadows=True, sun=sun, nthreads=NT)
        compare(g[i], o, shadows=True, what="sun %s cam %d" % (sun, i))


def test_repair_after_edits_equals_a_fresh_build(hf):
    cells = _world(9, 300, 220)
    sun = SUNS[0]
    rng = np.random.default_rng(5)
    ctx = hf.hf_create(cells)
    try:
        _bounds(hf, ctx, sun)
        for k in range(12):
            cx, cy = int(rng.integers(0, 300)), int(rng.integers(0, 220))
            x0, y0, blk = synth.crater_edit(cells, cx, cy)
            if k % 4 == 3:  # a tall block: shadows reach far
                blk = np.full_like(blk, synth.pack_cells(230, 0, 0, 2))
            hf.hf_edit(ctx, x0, y0, blk)
            cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
        hf.hf_sync(ctx)
        got, _ = hf.hf_read_sun_bounds(ctx)
        cams = synth.c3_cameras(cells, seed=8, n=6, scale=24)
        g = gpu_render(hf, ctx, cams, shadows=True)
    finally:
        hf.hf_destroy(ctx)
    fresh = hf.hf_create(cells)
    try:
        want = _bounds(hf, fresh, sun)
    finally:
        hf.hf_destroy(fresh)
    assert np.array_equal(got, want)
    for i, c in enumerate(cams):
        compare(g[i], oracle.render(cells, c, shadows=True, nthreads=NT), shadows=True,
                what="after edits cam %d" % i)


def test_alternating_suns_rebuild_the_bounds(hf):
    cfg = synth.config_c3(scale=32)
    cells, cams = cfg["cells"], cfg["cams"][:8]
    ctx = hf.hf_create(cells)
    try:
        for sun in (SUNS[0], SUNS[3], SUNS[0], NO_BOUNDS[0], SUNS[3]):
            g = gpu_render(hf, ctx, cams, shadows=True,
                           opts=hf.make_opts(flags=hf.HF_SHADOWS, sun=sun))
            for i, c in enumerate(cams):
                o = oracle.render(cells, c, shadows=True, sun=sun, nthreads=NT)
                compare(g[i], o, shadows=True, what="sun %s cam %d" % (sun, i))
    finally:
        hf.hf_destroy(ctx)


def test_bounds_cut_shadow_fetches(hf):
    """The fetch counters with the bounds: most shadow rays of the batched
    workload are decided by one lookup."""
    cfg = synth.config_c3(scale=8)
    cells, cams = cfg["cells"], cfg["cams"]
    ctx = hf.hf_create(cells)
    try:
        hf.hf_stats(ctx)
        gpu_render(hf, ctx, cams, shadows=True,
                   opts=hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_STATS))
        with_b = hf.hf_stats(ctx)
        low = (320000, 0, 5000)  # no bounds for this sun
        gpu_render(hf, ctx, cams, shadows=True,
                   opts=hf.make_opts(flags=hf.HF_SHADOWS | hf.HF_STATS, sun=low))
        without = hf.hf_stats(ctx)
    finally:
        hf.hf_destroy(ctx)
    assert with_b["shadow_rays"] > 0.5 * with_b["rays"]
    per_shadow = with_b["shadow_fetches"] / with_b["shadow_rays"]
    assert per_shadow < 8.0, per_shadow
    assert without["shadow_fetches"] / without["shadow_rays"] > per_shadow


def test_shadowed_renders_on_two_streams_around_an_edit(hf):
    """A shadowed render on one stream, then an edit (a tall block whose
    shadow reaches far upstream, so the bounds of many cells change), then a
    shadowed render on another stream: the first sees the old world, the
    second the new one, each equal to the oracle."""
    import torch

    cfg = synth.config_c1()
    cells = cfg["cells"].copy()
    cams = cfg["cams"]
    ctx = hf.hf_create(cells)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        a = hf.alloc_outputs(cams, shadows=True)
        hf.hf_render(ctx, cams, a, hf.make_opts(flags=hf.HF_SHADOWS, stream=s1.cuda_stream))
        blk = np.full((20, 20), synth.pack_cells(250, 0, 0, 3), np.uint32)
        hf.hf_edit(ctx, 150, 90, blk)
        cells[90:110, 150:170] = blk
        b = hf.alloc_outputs(cams, shadows=True)
        hf.hf_render(ctx, cams, b, hf.make_opts(flags=hf.HF_SHADOWS, stream=s2.cuda_stream))
        hf.hf_sync(ctx)
        torch.cuda.synchronize()
        fix = lambda o: {k: (v.cpu().numpy().view(np.uint32) if k in ("hit_cell", "rgba")
                             else v.cpu().numpy()) for k, v in o.items()}
        compare(fix(a[0]), oracle.render(cfg["cells"], cams[0], shadows=True), shadows=True,
                what="stream 1 before the edit")
        compare(fix(b[0]), oracle.render(cells, cams[0], shadows=True), shadows=True,
                what="stream 2 after the edit")
        fa, fb = fix(a[0]), fix(b[0])
        assert any((fa[k] != fb[k]).any() for k in ("shadow", "hit_cell"))  # the edit shows
    finally:
        hf.hf_destroy(ctx)


def test_native_serving_loop_with_shadow_rays(hf):
    """hf_serve_replay with HF_SHADOWS: renders on several lanes in flight,
    crater edits repairing the shadow bounds in between; every served image
    equals the oracle on the world with exactly the edits before it."""
    import torch

    cells, _ = synth.make_grid(384, 384, seed=23, slab_frac=0.3, n_walls=16)
    records = synth.poisson_requests(cells, 40, rate=2e4, seed=4, edit_every=5,
                                     resolutions=((96, 64), (160, 90), (64, 48)))
    outs = [None if r["kind"] == "edit" else hf.alloc_outputs(np.array([r["cam"]]),
                                                              shadows=True)[0]
            for r in records]
    ctx = hf.hf_create(cells)
    try:
        res = hf.hf_serve_replay(ctx, records, lanes=4, max_batch=3, output_budget=64 << 20,
                                 flags=hf.HF_SHADOWS, outputs=outs)
        hf.hf_sync(ctx)
        torch.cuda.synchronize()
    finally:
        hf.hf_destroy(ctx)
    assert len(set(res["batch"][res["batch"] != 0xFFFFFFFF])) > 3
    world = cells.copy()
    checked = 0
    for i, rec in enumerate(records):
        if rec["kind"] == "edit":
            x0, y0, blk = rec["edit"]
            world[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
            continue
        g = {k: (v.cpu().numpy().view(np.uint32) if k in ("hit_cell", "rgba") else v.cpu().numpy())
             for k, v in outs[i].items()}
        compare(g, oracle.render(world, rec["cam"], shadows=True), shadows=True,
                what="served request %d" % i)
        checked += 1
    assert checked == sum(r["kind"] == "render" for r in records)
