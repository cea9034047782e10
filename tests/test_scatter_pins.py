"""Pins of the scatter oracle (no GPU): its projection against exact rational
arithmetic, its footprint warp, its column walk, nearest-wins packing, a
closed-form depth, and agreement with the exact cast at a high density."""

from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import scatter
from paper_2608_17390_gb300 import metrics
from synth.scatter import footprint_for

f32 = np.float32


def test_projection_matches_exact_rationals():
    """A point's pixel from the float32 projection equals the pixel whose
    frustum holds it in exact arithmetic (a = (v.R/|R|^2) / (v.F/|F|^2) of the
    camera model d = F + aR + bU), away from pixel boundaries."""
    rng = np.random.default_rng(4)
    cams = [synth.config_c1()["cams"][0],
            synth.camera_array([synth.pose_to_camera(30.0, 40.0, 80.0, 200.0, -60.0, 75, 97, 55)])[0],
            synth.camera_array([synth.pose_to_camera(300.5, 10.0, 12.0, 45.0, 5.0, 90, 64, 32)])[0]]
    checked = 0
    for cam in cams:
        k = scatter.camera_constants(cam)
        F, R, U = (np.asarray(cam[x], np.int64) for x in ("f", "r", "u"))
        w, h = int(cam["w"]), int(cam["h"])
        O = [Fraction(int(o), 65536) for o in cam["o"]]
        for _ in range(400):
            a0 = rng.uniform(-(w - 1), w - 1)
            b0 = rng.uniform(-(h - 1), h - 1)
            d = F + a0 * R + b0 * U
            lam = rng.uniform(0.5, 40.0) / np.linalg.norm(d)
            P = np.array([float(O[i]) + lam * d[i] for i in range(3)], dtype=f32)
            pix, _ = scatter._project(k, P[0:1], P[1:2], P[2:3], 4096.0)
            v = [Fraction(float(P[i])) - O[i] for i in range(3)]
            dot = lambda V: sum(v[i] * int(V[i]) for i in range(3))
            nn = lambda V: sum(int(V[i]) ** 2 for i in range(3))
            a = (dot(R) / nn(R)) / (dot(F) / nn(F))
            b = (dot(U) / nn(U)) / (dot(F) / nn(F))
            xa, xb = (a + w) / 2, (h - b) / 2
            if min(abs(xa - round(xa)), abs(xb - round(xb))) < Fraction(1, 1000):
                continue  # too close to a pixel edge for float32
            px, py = int(np.floor(float(xa))), int(np.floor(float(xb)))
            want = py * w + px if (0 <= px < w and 0 <= py < h) else -1
            assert int(pix[0]) == want, (a, b, pix)
            checked += 1
    assert checked > 1000


def test_footprint_warp_crowds_samples_near_the_camera():
    cam = synth.config_c1()["cams"][0]
    k = scatter.camera_constants(cam)
    x, y = scatter.footprint(k, 8, 64, -2.0, 300.0, 0.5, 3.0)
    s = (x - k["Of"][0]) * k["fh"][0] + (y - k["Of"][1]) * k["fh"][1]
    col = s[:, 4].astype(np.float64)
    gaps = np.diff(col)
    assert (gaps > 0).all() and (np.diff(gaps) > 0).all()  # spacing grows with distance
    assert abs(col[0] - (-2.0 + 302.0 * (0.5 / 64) ** 2)) < 1e-3
    assert abs(col[-1] - (-2.0 + 302.0 * (63.5 / 64) ** 2)) < 1e-2
    u = (x - k["Of"][0]) * k["rh"][0] + (y - k["Of"][1]) * k["rh"][1]
    half = 3.0 + np.abs(col) * 0.5
    assert np.allclose(np.abs(u[:, [0, 7]]).max(axis=1), half * (7 / 8), rtol=1e-4, atol=1e-3)


def _grid(W, H, h0=0):
    return np.full((H, W), synth.pack_cells(h0, 0, 0, 0), np.uint32)


def test_column_walk_spans_floor_to_zero_and_slab_top_to_underside():
    """A lone column seen from the side covers exactly the image rows its
    walked points project to: from its top (h0) down to z = 0, and for a slab
    from h2 down to h1."""
    cells = _grid(64, 64)
    cells[32, 40] = synth.pack_cells(20, 0, 0, 3)
    cells[32, 44] = synth.pack_cells(2, 30, 36, 5)
    cam = synth.camera_array([synth.pose_to_camera(20.5, 32.5, 18.0, 90.0, 0.0, 60, 41, 41)])[0]
    out = scatter.render(cells, cam, 256, 512, 41, 0.0, 40.0, 0.6, 2.0, 256.0)
    k = scatter.camera_constants(cam)
    mat = out["material"].reshape(41, 41)
    layer = out["layer"].reshape(41, 41)
    for cx, z0, z1, m, lay in ((40, 20.0, 0.0, 3, 0), (44, 36.0, 30.0, 5, 1)):
        # image rows of the column's extreme points (front and back faces),
        # clipped into the image
        rows = []
        for z in (z0, z1):
            for x in (cx, cx + 1.0):
                v = np.array([x, 32.5, z], np.float64) - k["Of"].astype(np.float64)
                F, U = k["F"].astype(np.float64), k["U"].astype(np.float64)
                b = (v @ U / (U @ U)) / (v @ F / (F @ F))
                rows.append(int(min(40, max(0, np.floor((41 - b) / 2)))))
        rows.sort()
        hit_rows = {r for r in range(41) if ((mat[r] == m) & (layer[r] == lay)).any()}
        assert hit_rows, m
        assert min(hit_rows) <= rows[0] + 1 and max(hit_rows) >= rows[-1] - 1, (m, rows, hit_rows)
        assert min(hit_rows) >= rows[0] - 1 and max(hit_rows) <= rows[-1] + 1, (m, rows, hit_rows)


def test_nearest_point_wins_the_pixel():
    """Two walls one behind the other: the screen of both is the elementwise
    minimum of each wall's own screen, and where both reach a pixel the nearer
    one's material is kept (the packed word orders by depth first)."""
    near, far = _grid(64, 64), _grid(64, 64)
    near[20:44, 30] = synth.pack_cells(40, 0, 0, 2)
    far[10:54, 34] = synth.pack_cells(60, 0, 0, 6)
    both = np.maximum(near, far)  # (heights only in one of them per cell)
    cam = synth.camera_array([synth.pose_to_camera(10.5, 32.0, 20.0, 90.0, 0.0, 70, 48, 32)])[0]
    args = (cam, 512, 512, 48, 0.0, 40.0, 0.8, 2.0, 128.0)
    pn, pf, pb = (scatter.scatter_buffer(g, *args) for g in (near, far, both))
    assert (pb == np.minimum(pn, pf)).all()
    shared = (pn != scatter.EMPTY) & (pf != scatter.EMPTY)
    assert shared.sum() > 50
    qn, qf = pn[shared] >> 8, pf[shared] >> 8
    mat = pb[shared] & 7
    assert ((qn < qf) == (mat == 2)).all() and (qn < qf).mean() > 0.9


def test_depth_of_a_flat_plane_seen_from_above():
    """Camera H units above a flat plane h0 = c, looking straight down: the
    centre pixel's depth is H - c within the depth quantum plus the sampling
    offset of the nearest footprint sample."""
    c, H = 10, 50.0
    cells = _grid(128, 128, c)
    cam = synth.camera_array([synth.pose_to_camera(64.0, 64.0, H, 0.0, -90.0, 60, 33, 33)])[0]
    fp = footprint_for(cam)
    out = scatter.render(cells, cam, 1024, 1024, 2, *fp, 256.0)
    dc = float(out["depth"][16 * 33 + 16])
    assert abs(dc - (H - c)) < 0.05, dc
    hit = out["layer"] != 255
    assert hit.mean() > 0.99
    assert (out["depth"][hit] >= (H - c) - 1e-3).all()


def test_agrees_with_the_exact_cast_at_high_density():
    cfg = synth.config_c1()
    cells, cam = cfg["cells"], cfg["cams"][0]
    out = scatter.render(cells, cam, 1024, 2048, 32, *footprint_for(cam), 1024.0)
    ex = oracle.render(cells, cam)
    w, h = int(cam["w"]), int(cam["h"])
    m = metrics.compare((ex["layer"] != 255).reshape(h, w), ex["depth"].reshape(h, w),
                        (out["layer"] != 255).reshape(h, w), out["depth"].reshape(h, w))
    assert m["see_through"] < 0.002 and m["geometry_median"] < 0.5, m
    both = (ex["layer"] != 255) & (out["layer"] != 255)
    # where both see terrain, the reconstructed cell is the exact hit's cell or
    # a neighbour (a point near a cell edge, depth-quantised, may cross it)
    W = cells.shape[1]
    ea, oa = ex["hit_cell"][both].astype(np.int64), out["hit_cell"][both].astype(np.int64)
    cheb = np.maximum(np.abs(ea % W - oa % W), np.abs(ea // W - oa // W))
    assert (cheb <= 1).mean() > 0.8 and (cheb == 0).mean() > 0.5, ((cheb <= 1).mean(), (cheb == 0).mean())


MUTANTS = [
    ("linear footprint warp", "s = f32(s_lo) + (f32(s_hi) - f32(s_lo)) * (t * t)",
     "s = f32(s_lo) + (f32(s_hi) - f32(s_lo)) * t", "test_footprint_warp_crowds_samples_near_the_camera"),
    ("image rows flipped", "pyf = np.floor((f32(h) - b) * f32(0.5))",
     "pyf = np.floor((f32(h) + b) * f32(0.5))", "test_projection_matches_exact_rationals"),
    ("farthest point kept", "np.minimum.at(buf, pix[ok], packed[ok])",
     "np.maximum.at(buf, pix[ok], packed[ok])", "test_nearest_point_wins_the_pixel"),
    ("right and up swapped", "a = (vr * k[\"cR\"]) / den", "a = (vu * k[\"cU\"]) / den",
     "test_projection_matches_exact_rationals"),
    ("slab walked from the floor", "(1, h2 + (h1 - h2) * tm, slab)", "(1, h1 + (h0 - h1) * tm, slab)",
     "test_column_walk_spans_floor_to_zero_and_slab_top_to_underside"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS)
def test_pins_catch_planted_scatter_mistakes(name, old, new, pin, monkeypatch):
    import types

    src = open(scatter.__file__).read()
    assert src.count(old) == 1, name
    mutant = types.ModuleType("scatter_mutant")
    exec(compile(src.replace(old, new), "scatter_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "scatter", mutant)
    with pytest.raises(AssertionError):
        globals()[pin]()
