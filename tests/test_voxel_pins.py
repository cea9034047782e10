"""Pins of the RayVoxel oracle (no GPU): occupancy against a per-voxel loop,
the union levels, conservativeness, the Morton tile packing by hand, the
vectorised traversal against the one-ray form, independence of the starting
level, the paper's stated trade-off (a thin sheet slips between leaf samples),
closeness to the exact cast at fine voxels, and planted mistakes."""

import numpy as np
import pytest

import oracle
import synth
from oracle import voxel


def _rand_grid(rng, W, H, hmax=60):
    h0 = rng.integers(0, hmax, (H, W))
    slab = rng.random((H, W)) < 0.4
    h1 = np.where(slab, np.minimum(255, h0 + rng.integers(1, 40, (H, W))), 0)
    h2 = np.where(slab, np.minimum(255, h1 + rng.integers(0, 30, (H, W))), 0)
    return synth.pack_cells(h0, h1, h2, rng.integers(0, 8, (H, W)))


@pytest.mark.parametrize("v", [(4, 8, 2), (1, 1, 1), (3, 5, 7), (8, 8, 16)])
def test_level0_occupancy_equals_the_per_voxel_loop(v):
    rng = np.random.default_rng(sum(v))
    cells = _rand_grid(rng, 13, 11, hmax=200)
    assert np.array_equal(voxel.level0(cells, *v), voxel.level0_loop(cells, *v))


def test_levels_are_unions_of_their_children():
    rng = np.random.default_rng(2)
    cells = _rand_grid(rng, 37, 29)
    lv = voxel.pyramid(cells, 2, 3, 4, 5)
    for k in range(1, 5):
        a, b = lv[k - 1], lv[k]
        for z in range(b.shape[0]):
            for y in range(b.shape[1]):
                for x in range(b.shape[2]):
                    want = a[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2].any()
                    assert b[z, y, x] == want


def test_every_solid_point_lies_in_occupied_voxels_at_every_level():
    rng = np.random.default_rng(3)
    cells = _rand_grid(rng, 40, 30, hmax=120)
    g = voxel.Grid(cells, 4, 8, 2, 5)
    h0, h1, h2, _ = (a.astype(np.int64) for a in synth.unpack_cells(cells))
    for _ in range(3000):
        y, x = int(rng.integers(0, 30)), int(rng.integers(0, 40))
        px, py = x + rng.random(), y + rng.random()
        if h1[y, x] > h0[y, x] and rng.random() < 0.5:
            z = rng.uniform(h1[y, x], h2[y, x])
        else:
            z = rng.uniform(0, h0[y, x]) if h0[y, x] > 0 else 0.0
        i, j, k = int(px // 4), int(py // 8), int(z // 2)
        for l in range(5):
            assert g.levels[l][k >> l, j >> l, i >> l], (x, y, z, l)


def test_morton_bits_and_tile_packing_by_hand():
    assert [voxel.morton3(*p) for p in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (2, 0, 0),
                                         (0, 2, 0), (4, 0, 0), (7, 7, 7), (3, 5, 6)]] == \
        [1, 2, 4, 7, 8, 16, 64, 511, 0b110101011]
    lv = np.zeros((9, 17, 10), bool)  # nz, ny, nx: tiles TX = 2, TY = 3, TZ = 2
    lv[8, 16, 9] = True  # tile (1, 2, 1) = (1 * 3 + 2) * 2 + 1 = 11; local (1, 0, 0): bit 1
    lv[0, 0, 0] = True   # tile 0, bit 0
    lv[3, 5, 6] = True   # tile 0, local (6, 5, 3): morton 6 + 40 + 192 = 238 -> word 7 bit 14
    w = voxel.pack(lv)
    assert np.array_equal(w, voxel.pack_loop(lv))
    rnd = np.random.default_rng(1).random((19, 23, 17)) < 0.3
    assert np.array_equal(voxel.pack(rnd), voxel.pack_loop(rnd))
    assert w.size == 2 * 3 * 2 * 16
    want = np.zeros_like(w)
    want[11 * 16 + 0] |= 1 << 1
    want[0] |= 1
    want[7] |= 1 << 14
    assert np.array_equal(w, want)


def _cams(cells):
    H, W = cells.shape
    return synth.camera_array([
        synth.pose_to_camera(W / 2, 3.0, 150.0, 0.0, -35.0, 70, 48, 30),
        synth.pose_to_camera(10.5, H / 2, float((cells[H // 2, 10] & 0xFF) + 3), 80.0, -2.0, 90, 40, 20),
        synth.pose_to_camera(W / 2, H / 2, 300.0, 30.0, -90.0, 60, 32, 32),
        synth.pose_to_camera(W - 5.0, H - 5.0, 90.0, 225.0, 10.0, 60, 24, 16),
    ])


def test_vectorised_traversal_equals_the_one_ray_form_and_any_start_level():
    rng = np.random.default_rng(6)
    cells = _rand_grid(rng, 96, 80, hmax=150)
    for v, levels in (((4, 8, 2), 5), ((2, 2, 2), 6), ((5, 3, 4), 4)):
        g = voxel.Grid(cells, *v, levels)
        flat = voxel.Grid(cells, *v, 1)
        for cam in _cams(cells):
            dirs = oracle.ray_dirs(cam)
            out = voxel.trace(g, cam["o"], dirs, inner=3)
            out0 = voxel.trace(flat, cam["o"], dirs, inner=3)
            for k in ("hit_cell", "layer"):
                assert np.array_equal(out[k], out0[k]), (v, k)
            assert np.array_equal(out["depth"].view(np.uint32), out0["depth"].view(np.uint32))
            for i in range(0, len(dirs), 29):
                r = voxel.trace_one(g, cam["o"], dirs[i], inner=3)
                if r is None:
                    assert out["layer"][i] == 255
                else:
                    assert (out["hit_cell"][i], out["layer"][i]) == r[:2] and out["depth"][i] == r[2]


def test_only_occupied_voxels_are_entered_or_sampled():
    rng = np.random.default_rng(8)
    cells = _rand_grid(rng, 64, 64, hmax=90)
    g = voxel.Grid(cells, 4, 4, 4, 5)
    cam = _cams(cells)[0]
    dirs = oracle.ray_dirs(cam)
    for i in range(0, len(dirs), 53):
        visits = []
        voxel.trace_one(g, cam["o"], dirs[i], visits=visits)
        for (l, x, y, z, occ, t), nxt in zip(visits, visits[1:] + [None]):
            if occ and l > 0:  # an occupied node is always opened, never skipped
                assert nxt is not None and nxt[0] == l - 1 and nxt[5] == t
            if nxt is not None and nxt[0] == l + 1:  # a climb happens only after a step
                assert nxt[5] > t or not occ
        ts = [v[5] for v in visits]
        assert all(a <= b for a, b in zip(ts, ts[1:]))


def test_a_thin_sheet_slips_between_leaf_samples():
    """The paper's stated trade-off: fixed leaf sampling can miss a feature
    thinner than its sample spacing; the exact cast cannot."""
    cells = np.full((64, 64), synth.pack_cells(0, 0, 0, 0), np.uint32)
    cells[20:44, 20:44] = synth.pack_cells(0, 100, 100, 3)  # zero-thickness sheet at z = 100
    cam = synth.camera_array([synth.pose_to_camera(32.0, 5.0, 101.5, 0.0, -8.0, 40, 32, 24)])[0]
    dirs = oracle.ray_dirs(cam)
    ex = oracle.render(cells, cam)
    out = voxel.trace(voxel.Grid(cells, 4, 4, 2, 4), cam["o"], dirs, inner=4)
    sheet = ex["layer"] == 1
    assert sheet.sum() > 50
    assert (out["layer"][sheet] != 1).mean() > 0.9


def test_close_to_the_exact_cast_with_fine_voxels_and_dense_samples():
    cfg = synth.config_c1()
    cells, cam = cfg["cells"], cfg["cams"][0]
    out = voxel.trace(voxel.Grid(cells, 1, 1, 1, 7), cam["o"], oracle.ray_dirs(cam), far=2000.0,
                      inner=16)
    ex = oracle.render(cells, cam)
    both = (ex["layer"] != 255) & (out["layer"] != 255)
    assert both.mean() > 0.98
    assert (ex["hit_cell"][both] == out["hit_cell"][both]).mean() > 0.97
    err = np.abs(out["depth"][both].astype(np.float64) - ex["depth"][both])
    assert np.median(err) < 0.05


MUTANTS = [
    ("occupancy by intersection", ".any(axis=(1, 3, 5)))", ".all(axis=(1, 3, 5)))",
     "test_levels_are_unions_of_their_children"),
    ("open floor interval", "np.minimum(h0 // vz, nz0 - 1)", "np.minimum((h0 - 1) // vz, nz0 - 1)",
     "test_level0_occupancy_equals_the_per_voxel_loop"),
    ("climb on the wrong parity", "up[m] = np.where(sgn > 0, ia % 2 == 0, ia % 2 == 1)",
     "up[m] = np.where(sgn > 0, ia % 2 == 1, ia % 2 == 0)",
     "test_vectorised_traversal_equals_the_one_ray_form_and_any_start_level"),
    ("first child against the direction", "first = 2 * idx[a][rd] + (d[a][rd] < 0)",
     "first = 2 * idx[a][rd] + (d[a][rd] > 0)",
     "test_vectorised_traversal_equals_the_one_ray_form_and_any_start_level"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS)
def test_pins_catch_planted_voxel_mistakes(name, old, new, pin, monkeypatch):
    import types

    src = open(voxel.__file__).read()
    assert src.count(old) == 1, name
    mutant = types.ModuleType("voxel_mutant")
    exec(compile(src.replace(old, new), "voxel_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "voxel", mutant)
    caught = False
    try:
        if pin == "test_level0_occupancy_equals_the_per_voxel_loop":
            for v in [(4, 8, 2), (1, 1, 1), (3, 5, 7), (8, 8, 16)]:
                globals()[pin](v)
        else:
            globals()[pin]()
    except AssertionError:
        caught = True
    assert caught, name
