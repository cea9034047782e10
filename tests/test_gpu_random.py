"""Randomised differential tests against the oracle (GPU only).

Seeded random worlds of many shapes (strips one cell wide, odd sizes, grids
too small for the pyramid's coarse levels), random sun directions that have
shadow bounds and some that have none, random cameras, and random edits
(arbitrary valid cells, slabs included) between renders.  After every edit the
shadowed render must equal the oracle on the edited cells (hit cell, layer,
face and shadow exact; depth within 1e-5 relative; colour within 1/255), and
the shadow bounds repaired by the edits must equal a fresh build bit for bit.
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


@pytest.fixture(scope="module")
def hf():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    import paper_2608_17390_gb300 as m

    return m


def _cells(rng, W, H):
    h0 = rng.integers(0, 140, (H, W))
    walls = rng.random((H, W)) < 0.04
    h0 = np.where(walls, 200, h0)
    slab = (rng.random((H, W)) < rng.uniform(0.0, 0.6)) & ~walls
    h1 = np.where(slab, np.minimum(h0 + rng.integers(1, 40, (H, W)), 254), 0)
    h2 = np.where(slab, np.minimum(h1 + rng.integers(0, 30, (H, W)), 255), 0)
    slab = h1 > h0
    return synth.pack_cells(h0, np.where(slab, h1, 0), np.where(slab, h2, 0),
                            rng.integers(0, 8, (H, W)))


def _sun(rng, k):
    if k % 5 == 0:  # exactly diagonal or along an axis
        a = int(rng.integers(100000, 500000))
        sx, sy = int(rng.choice([-1, 1])), int(rng.choice([-1, 1]))
        return [(sx * a, sy * a, int(rng.integers(150000, 600000))),
                (sx * a, 0, int(rng.integers(150000, 600000))),
                (0, sy * a, int(rng.integers(150000, 600000)))][k % 3]
    if k % 7 == 3:  # one without bounds (low, or below the horizon)
        return (int(rng.integers(300000, 900000)), int(rng.integers(-90000, 90000)),
                int(rng.choice([-1, 1])) * int(rng.integers(1000, 20000)))
    lx, ly = (int(v) for v in rng.integers(-900000, 900000, 2))
    lz = int(rng.integers(60000, 900000))
    return (lx or 1, ly, lz)


def _cams(rng, W, H, n):
    cams = []
    for _ in range(n):
        x, y = float(rng.uniform(0.01, W - 0.01)), float(rng.uniform(0.01, H - 0.01))
        cams.append(synth.pose_to_camera(x, y, float(rng.uniform(1.0, 260.0)),
                                         float(rng.uniform(0, 360)), float(rng.uniform(-85, 20)),
                                         float(rng.uniform(40, 100)), 40, 28))
    return synth.camera_array(cams)


SHAPES = [(1, 1), (1, 37), (45, 1), (3, 70), (17, 17), (31, 33), (64, 64), (96, 40), (40, 96),
          (127, 65), (200, 3), (2, 150)]


@pytest.mark.parametrize("k", range(len(SHAPES) * 8))
def test_random_worlds_suns_and_edits_equal_the_oracle(hf, k):
    rng = np.random.default_rng(7000 + k)
    W, H = SHAPES[k % len(SHAPES)]
    cells = _cells(rng, W, H)
    sun = _sun(rng, k)
    cams = _cams(rng, W, H, 3)
    opts = hf.make_opts(flags=hf.HF_SHADOWS, sun=sun,
                        mip_start=int(rng.integers(0, 8)) if k % 3 else hf.HF_MIP_AUTO)
    ctx = hf.hf_create(cells)
    try:
        for step in range(3):
            g = gpu_render(hf, ctx, cams, shadows=True, opts=opts)
            for i, c in enumerate(cams):
                o = oracle.render(cells, c, shadows=True, sun=sun, nthreads=NT)
                compare(g[i], o, shadows=True,
                        what="world %dx%d sun %s step %d cam %d" % (W, H, sun, step, i))
            # an edit of random valid cells in a random rectangle
            ew, eh = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
            ew, eh = min(ew, 24), min(eh, 24)
            x0, y0 = int(rng.integers(0, W - ew + 1)), int(rng.integers(0, H - eh + 1))
            blk = _cells(rng, ew, eh)
            hf.hf_edit(ctx, x0, y0, blk)
            cells[y0:y0 + eh, x0:x0 + ew] = blk
        hf.hf_sync(ctx)
        try:
            got, s = hf.hf_read_sun_bounds(ctx)
        except hf.HFError:
            got = None  # this sun has no bounds
    finally:
        hf.hf_destroy(ctx)
    if got is not None:
        assert s == tuple(sun)
        fresh = hf.hf_create(cells)
        try:
            gpu_render(hf, fresh, cams[:1], shadows=True, opts=opts)
            want, _ = hf.hf_read_sun_bounds(fresh)
        finally:
            hf.hf_destroy(fresh)
        assert np.array_equal(got, want), "repaired bounds differ from a fresh build"
