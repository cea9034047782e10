"""Pins for the CPU oracle against things other than itself.

* hand-derived cases (tests/golden/hand_cases.json);
* the independent brute-force checker (oracle/brute.py) on random tiny grids
  with rays on a quarter-cell lattice, so exact corner, boundary and grazing
  ties are frequent;
* closed forms written here with exact fractions: a flat plane, one floating
  slab box over a flat floor, a vertical wall, and a wall's shadow;
* hand-derived colours for every face of a cell, lit, turned away from the
  sun and occluded (tests/golden/shading_faces.json);
* the pyramid against a second implementation and against the parent/child
  recurrence.
"""

import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

S = 65536
HERE = os.path.dirname(os.path.abspath(__file__))


def _grid(W, H, spec):
    h0 = np.zeros((H, W), np.int64)
    h1 = np.zeros((H, W), np.int64)
    h2 = np.zeros((H, W), np.int64)
    mat = np.zeros((H, W), np.int64)
    for x, y, a, b, c, m in spec:
        h0[y, x], h1[y, x], h2[y, x], mat[y, x] = a, b, c, m
    return synth.pack_cells(h0, h1, h2, mat)


def _rand_grid(rng, W, H, hmax=12):
    h0 = rng.integers(0, hmax, (H, W))
    slab = rng.random((H, W)) < 0.4
    h1 = np.where(slab, h0 + rng.integers(1, 6, (H, W)), 0)
    h2 = np.where(slab, h1 + rng.integers(0, 5, (H, W)), 0)
    return synth.pack_cells(h0, h1, h2, rng.integers(0, 8, (H, W)))


def _same(b, r, k, W):
    depth_ok = (b[3] == r["depth"][k]) or abs(b[3] - r["depth"][k]) <= 1e-12 * abs(b[3])
    return (b[0] == r["hit_cell"][k] and b[1] == r["layer"][k] and b[2] == r["face"][k]
            and depth_ok)


# --------------------------------------------------------------- hand cases

def _hand_cases():
    with open(os.path.join(HERE, "golden", "hand_cases.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_hand_case(case):
    cells = _grid(4, 4, case["cells"])
    o = np.array([[round(v * S) for v in case["origin"]]], np.int64)
    d = np.array([[round(v * S) for v in case["dir"]]], np.int64)
    e = case["expect"]
    cell = 0xFFFFFFFF if e["x"] < 0 else e["y"] * 4 + e["x"]
    depth = math.inf if e["depth"] == "inf" else e["depth"]
    for impl in ("oracle", "brute"):
        if impl == "oracle":
            r = oracle.trace_rays(cells, o, d)
            got = (int(r["hit_cell"][0]), int(r["layer"][0]), int(r["face"][0]), float(r["depth"][0]))
        else:
            got = brute.trace(cells, o[0], d[0])
        assert got[:3] == (cell, e["layer"], e["face"]), (impl, got)
        if math.isinf(depth):
            assert math.isinf(got[3])
        else:
            assert got[3] == pytest.approx(depth, rel=1e-12, abs=1e-12), impl


# --------------------------------------------------------- oracle vs brute

def _lattice_rays(rng, W, H, n):
    o = np.stack([rng.integers(0, 4 * W, n) * S // 4, rng.integers(0, 4 * H, n) * S // 4,
                  rng.integers(0, 64, n) * S // 4], 1)
    d = np.stack([rng.integers(-4, 5, n) * S // 4, rng.integers(-4, 5, n) * S // 4,
                  rng.integers(-4, 5, n) * S // 8], 1)
    k = n // 6
    o[:k] = np.stack([rng.integers(0, W * S, k), rng.integers(0, H * S, k),
                      rng.integers(0, 16 * S, k)], 1)
    d[:k] = rng.integers(-S, S, (k, 3))
    return o.astype(np.int64), d.astype(np.int64)


def test_oracle_matches_brute_on_tiny_grids():
    rng = np.random.default_rng(1234)
    seen_faces = set()
    mism = []
    for _ in range(40):
        W, H = int(rng.integers(3, 10)), int(rng.integers(3, 10))
        cells = _rand_grid(rng, W, H)
        o, d = _lattice_rays(rng, W, H, 60)
        r = oracle.trace_rays(cells, o, d)
        for k in range(len(o)):
            b = brute.trace(cells, o[k], d[k])
            seen_faces.add(b[2])
            if not _same(b, r, k, W):
                mism.append((W, H, o[k].tolist(), d[k].tolist(), b))
    assert not mism, mism[:5]
    # the sample must exercise every face code and misses
    assert seen_faces >= {0, 1, 2, 3, 4, 5, 6, 255}, seen_faces


def test_oracle_matches_brute_on_camera_rays():
    """Rays from the integer camera model d = F + (2px+1-w)R + (h-1-2py)U."""
    rng = np.random.default_rng(77)
    cells = _rand_grid(rng, 12, 10, hmax=30)
    cam = synth.camera_array([synth.pose_to_camera(2.5, 1.25, 20.0, 30.0, -40.0, 70.0, 9, 7)])[0]
    r = oracle.render(cells, cam)
    dirs = oracle.ray_dirs(cam)
    o = np.array(cam["o"], np.int64)
    bad = [k for k in range(len(dirs)) if not _same(brute.trace(cells, o, dirs[k]), r, k, 12)]
    assert not bad
    assert (r["face"] != 255).sum() > 0


def test_special_rays_match_brute():
    """Vertical rays, a zero direction, rays along column boundaries, rays
    starting on boundaries, grazing rays at exact heights."""
    rng = np.random.default_rng(5)
    cells = _rand_grid(rng, 6, 6, hmax=8)
    rays = []
    for x in (0, S // 2, S, 3 * S, 6 * S - 1):
        for z in (0, 3 * S, 8 * S, 20 * S):
            rays.append(((x, 2 * S, z), (0, 0, -S)))
            rays.append(((x, 2 * S, z), (0, 0, S)))
            rays.append(((x, 2 * S, z), (0, 0, 0)))
            rays.append(((x, 3 * S, z), (0, S, 0)))
            rays.append(((x, 3 * S, z), (0, -S, -S // 7)))
            rays.append(((x, 3 * S, z), (-S, 0, 0)))
            rays.append(((x, 3 * S, z), (S, S, -S // 3)))
            rays.append(((x, 3 * S, z), (-S, -S, S // 5)))
    o = np.array([r[0] for r in rays], np.int64)
    d = np.array([r[1] for r in rays], np.int64)
    res = oracle.trace_rays(cells, o, d)
    bad = [k for k in range(len(rays)) if not _same(brute.trace(cells, o[k], d[k]), res, k, 6)]
    assert not bad, [rays[k] for k in bad[:5]]


# ------------------------------------------------------------- closed forms

def _left_cell(p, d):
    """Cell the ray occupies just before reaching point p (exact fractions)."""
    c = math.floor(p / S)
    if d > 0 and p == c * S:
        c -= 1
    return c


def _right_cell(p, d):
    """Cell the ray occupies just after point p."""
    c = math.floor(p / S)
    if d < 0 and p == c * S:
        c -= 1
    return c


def test_closed_form_flat_plane():
    """Flat floor h0 = c: a descending ray from above hits the +Z face at
    t = (c S - oz)/dz, in the cell it occupies just before that point; rays
    that do not descend miss."""
    W = H = 24
    c = 37
    cells = _grid(W, H, [(x, y, c, 0, 0, (x + y) % 8) for x in range(W) for y in range(H)])
    rng = np.random.default_rng(9)
    n = 400
    o = np.stack([rng.integers(0, W * S, n), rng.integers(0, H * S, n),
                  rng.integers(c * S + 1, 80 * S, n)], 1).astype(np.int64)
    d = rng.integers(-S, S, (n, 3)).astype(np.int64)
    d[:40, 2] = 0
    d[40:60, 0] = 0
    r = oracle.trace_rays(cells, o, d)
    for k in range(n):
        ox, oy, oz = (int(v) for v in o[k])
        dx, dy, dz = (int(v) for v in d[k])
        if dz >= 0:
            assert r["face"][k] == 255
            continue
        t = Fr(c * S - oz, dz)
        px, py = ox + t * dx, oy + t * dy
        cx, cy = _left_cell(px, dx), _left_cell(py, dy)
        if not (0 <= cx < W and 0 <= cy < H):
            assert r["face"][k] == 255, k
            continue
        assert (r["hit_cell"][k], r["layer"][k], r["face"][k]) == (cy * W + cx, 0, 5), k
        depth = float(t) * math.sqrt(dx * dx + dy * dy + dz * dz) / S
        assert r["depth"][k] == pytest.approx(depth, rel=1e-12)


def _box_entry(o, d, lo, hi):
    """Slab method on a closed box: (t_enter, axis) or None.  Ties between
    axes go to x, then y, then z."""
    t0, t1, axis = Fr(0), None, None
    for a in range(3):
        if d[a] == 0:
            if not (lo[a] <= o[a] <= hi[a]):
                return None
            continue
        ta, tb = Fr(lo[a] - o[a], d[a]), Fr(hi[a] - o[a], d[a])
        if ta > tb:
            ta, tb = tb, ta
        if ta > t0 or (axis is None and ta == t0 and t0 > 0):
            t0, axis = ta, a
        t1 = tb if t1 is None else min(t1, tb)
    if t1 is not None and t0 > t1:
        return None
    return t0, axis


def test_closed_form_floating_slab():
    """One slab [h1, h2] over the cells [a, b) x [c, e) above a floor of 0:
    the first contact is the entry into the closed box (side faces win ties
    with the top, x wins ties with y), else the floor."""
    W, H = 20, 16
    a, b, c, e, h1, h2 = 6, 13, 4, 11, 9, 15
    spec = [(x, y, 0, h1, h2, 3) for x in range(a, b) for y in range(c, e)]
    cells = _grid(W, H, spec)
    rng = np.random.default_rng(21)
    n = 600
    o = np.stack([rng.integers(0, W * S, n), rng.integers(0, H * S, n),
                  rng.integers(1, 30 * S, n)], 1).astype(np.int64)
    d = rng.integers(-S, S, (n, 3)).astype(np.int64)
    d[: 2 * n // 3, 2] = -np.abs(d[: 2 * n // 3, 2]) - S // 2
    d[d == 0] = 1
    inside = ((o[:, 0] >= a * S) & (o[:, 0] <= b * S) & (o[:, 1] >= c * S) & (o[:, 1] <= e * S)
              & (o[:, 2] >= h1 * S) & (o[:, 2] <= h2 * S))
    o, d = o[~inside], d[~inside]
    r = oracle.trace_rays(cells, o, d)
    lo, hi = (a * S, c * S, h1 * S), (b * S, e * S, h2 * S)
    checked = 0
    for k in range(len(o)):
        ok_ = [int(v) for v in o[k]]
        dk = [int(v) for v in d[k]]
        hits = []
        ent = _box_entry(ok_, dk, lo, hi)
        if ent is not None:
            t, axis = ent
            p = [ok_[i] + t * dk[i] for i in range(3)]
            if axis == 2:
                cx, cy = _left_cell(p[0], dk[0]), _left_cell(p[1], dk[1])
                face = 5 if dk[2] < 0 else 4
            else:
                cx, cy = _right_cell(p[0], dk[0]), _right_cell(p[1], dk[1])
                face = (0 if dk[0] > 0 else 1) if axis == 0 else (2 if dk[1] > 0 else 3)
            hits.append((t, cy * W + cx, 1, face, (cx, cy)))
        if dk[2] < 0:
            t = Fr(-ok_[2], dk[2])
            p = [ok_[i] + t * dk[i] for i in range(2)]
            cx, cy = _left_cell(p[0], dk[0]), _left_cell(p[1], dk[1])
            hits.append((t, cy * W + cx, 0, 5, (cx, cy)))
        hits.sort(key=lambda h: h[0])
        exp = None
        if hits:
            t, cell, layer, face, (cx, cy) = hits[0]
            # the path to the contact point must stay in the grid
            if 0 <= cx < W and 0 <= cy < H:
                exp = (cell, layer, face)
        if exp is None:
            assert r["face"][k] == 255, (ok_, dk, r["hit_cell"][k], r["face"][k])
        else:
            assert (int(r["hit_cell"][k]), int(r["layer"][k]), int(r["face"][k])) == exp, (ok_, dk)
            checked += 1
    assert checked > 150


def test_closed_form_vertical_wall():
    """A one-column wall (h0 = 200) at column i over a floor of 0: a
    horizontal ray below 200 hits its -X face at t = (i S - ox)/dx when moving
    +x, its +X face at t = ((i+1) S - ox)/dx when moving -x."""
    W, H, i = 30, 12, 17
    cells = _grid(W, H, [(i, y, 200, 0, 0, 2) for y in range(H)])
    rng = np.random.default_rng(3)
    n = 300
    left = rng.random(n) < 0.5
    ox = np.where(left, rng.integers(0, i * S, n), rng.integers((i + 1) * S, W * S, n))
    dx = np.where(left, rng.integers(1, S, n), -rng.integers(1, S, n))
    o = np.stack([ox, rng.integers(0, H * S, n), rng.integers(1, 200 * S, n)], 1).astype(np.int64)
    d = np.stack([dx, rng.integers(-S // 8, S // 8, n), np.zeros(n, np.int64)], 1).astype(np.int64)
    r = oracle.trace_rays(cells, o, d)
    for k in range(n):
        oxk, oyk = int(o[k, 0]), int(o[k, 1])
        dxk, dyk = int(d[k, 0]), int(d[k, 1])
        bx = i * S if dxk > 0 else (i + 1) * S
        t = Fr(bx - oxk, dxk)
        py = oyk + t * dyk
        cy = _right_cell(py, dyk)
        if not (0 <= cy < H):
            assert r["face"][k] == 255
            continue
        face = 0 if dxk > 0 else 1
        assert (int(r["hit_cell"][k]), int(r["face"][k]), int(r["layer"][k])) == (cy * W + i, face, 0)
        assert r["depth"][k] == pytest.approx(float(t) * math.hypot(dxk, dyk) / S, rel=1e-12)


def test_closed_form_wall_shadow():
    """Floor of height 1 with a block of height 60: a floor hit is shadowed
    exactly when the shadow ray from one unit above the hit point, toward the
    sun, enters the block's closed box before leaving the grid."""
    W, H = 40, 40
    bx0, bx1, by0, by1, bh = 14, 18, 20, 24, 60
    spec = [(x, y, 1, 0, 0, 1) for x in range(W) for y in range(H)]
    spec = [s for s in spec if not (bx0 <= s[0] < bx1 and by0 <= s[1] < by1)]
    spec += [(x, y, bh, 0, 0, 4) for x in range(bx0, bx1) for y in range(by0, by1)]
    cells = _grid(W, H, spec)
    L = oracle.DEFAULT_SUN
    rng = np.random.default_rng(8)
    n = 500
    # vertical rays onto the floor: hit point (ox, oy, S), exact
    o = np.stack([rng.integers(0, W * S, n), rng.integers(0, H * S, n),
                  np.full(n, 100 * S)], 1).astype(np.int64)
    on_block = ((o[:, 0] >= bx0 * S) & (o[:, 0] < bx1 * S) & (o[:, 1] >= by0 * S) & (o[:, 1] < by1 * S))
    o = o[~on_block]
    d = np.tile(np.array([0, 0, -S], np.int64), (len(o), 1))
    r = oracle.trace_rays(cells, o, d, shadows=True)
    shadowed = 0
    for k in range(len(o)):
        p = [int(o[k, 0]), int(o[k, 1]), S + 1]
        ent = _box_entry(p, L, (bx0 * S, by0 * S, 0), (bx1 * S, by1 * S, bh * S))
        exp = 0
        if ent is not None:
            t = ent[0]
            q = [p[a] + t * L[a] for a in range(2)]
            if 0 <= q[0] <= W * S and 0 <= q[1] <= H * S:
                exp = 1
        assert r["face"][k] == 5
        assert int(r["shadow"][k]) == exp, (p, ent)
        shadowed += exp
    assert 10 < shadowed < len(o) - 10


def _shading_fixture():
    with open(os.path.join(HERE, "golden", "shading_faces.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _shading_fixture()["cases"], ids=lambda c: c["name"])
def test_shading_per_face(case):
    """One hand-derived colour per face of the cell, lit, turned away from
    the sun and occluded (tests/golden/shading_faces.json): pins the sign and
    axis of N.L for every face, the ambient and diffuse weights, the shadow
    factor and the rounding."""
    fx = _shading_fixture()
    W = H = 16
    h0 = np.full((H, W), 2, np.int64)
    h1 = np.zeros((H, W), np.int64)
    h2 = np.zeros((H, W), np.int64)
    mat = np.zeros((H, W), np.int64)
    for x0, x1, y0, y1, a, b, c, m in fx["scenes"][case["scene"]]:
        h0[y0:y1, x0:x1], h1[y0:y1, x0:x1], h2[y0:y1, x0:x1], mat[y0:y1, x0:x1] = a, b, c, m
    cells = synth.pack_cells(h0, h1, h2, mat)
    o = np.array([[round(v * S) for v in case["origin"]]], np.int64)
    d = np.array([case["dir"]], np.int64)
    r = oracle.trace_rays(cells, o, d, shadows=True, sun=tuple(fx["suns"][case["sun"]]))
    e = case["expect"]
    assert int(r["hit_cell"][0]) == e["y"] * W + e["x"]
    assert (int(r["layer"][0]), int(r["face"][0])) == (e["layer"], e["face"])
    assert float(r["depth"][0]) == pytest.approx(e["depth"], rel=1e-12)
    assert int(r["shadow"][0]) == e["shadow"]
    rgba = int(r["rgba"][0])
    assert [rgba & 0xFF, (rgba >> 8) & 0xFF, (rgba >> 16) & 0xFF, rgba >> 24] == e["rgb"] + [255]


def test_shading_invariants():
    """Misses get the sky colour; inside hits and shadowed hits get ambient
    light only; a face turned away from the sun gets ambient light only."""
    W = H = 8
    cells = _grid(W, H, [(x, y, 2, 0, 0, 5) for x in range(W) for y in range(H)])
    o = np.array([[S * 4, S * 4, S * 2], [S * 4, S * 4, S * 5], [S * 4, S * 4, S * 5]], np.int64)
    d = np.array([[S, 0, 0], [0, 0, S], [0, 0, -S]], np.int64)
    r = oracle.trace_rays(cells, o, d, shadows=True)
    assert r["face"].tolist() == [6, 255, 5]
    ambient = [math.floor(255 * a * 0.3 + 0.5) for a in (0.70, 0.35, 0.20)]
    amb = ambient[0] | (ambient[1] << 8) | (ambient[2] << 16) | (255 << 24)
    assert int(r["rgba"][0]) == amb
    assert int(r["rgba"][1]) == 0xFFEBB487
    lit = int(r["rgba"][2])
    assert lit != amb and (lit >> 24) == 255


# ----------------------------------------------------------------- pyramid

@pytest.mark.parametrize("W,H", [(1, 1), (2, 3), (7, 5), (16, 16), (33, 17), (64, 9), (100, 1)])
def test_pyramid_two_implementations(W, H):
    rng = np.random.default_rng(W * 1000 + H)
    cells = _rand_grid(rng, W, H, hmax=200)
    a = oracle.pyramid(cells)
    b = brute.pyramid(cells)
    assert len(a) == len(b) == oracle.levels_for(W, H)
    for x, y in zip(a, b):
        assert x.shape == y.shape and (x == y).all()


def test_pyramid_recurrence():
    """Each node equals the combination of its (up to four) children."""
    rng = np.random.default_rng(11)
    cells = _rand_grid(rng, 37, 29, hmax=200)
    levels = oracle.pyramid(cells)
    h0, h1, h2, _ = synth.unpack_cells(cells)
    slab = h1 > h0
    prev = (h0, np.where(slab, h1, 255), np.where(slab, h2, h0))
    for lv in levels:
        hk, wk = lv.shape
        for j in range(hk):
            for i in range(wk):
                sl = (slice(2 * j, 2 * j + 2), slice(2 * i, 2 * i + 2))
                e = (prev[0][sl].max(), prev[1][sl].min(), prev[2][sl].max())
                v = int(lv[j, i])
                assert (v & 0xFF, (v >> 8) & 0xFF, (v >> 16) & 0xFF) == e
        prev = (lv & 0xFF, (lv >> 8) & 0xFF, (lv >> 16) & 0xFF)
    assert levels[-1].shape == (1, 1)


def test_top_of_range_heights_match_brute():
    """Cells at the top of the height range (255) hit by rays at or just
    above z = 255 S: the rule that a non-descending ray above every cell
    misses must not cut these off."""
    W, H = 8, 5
    spec = [(5, y, 255, 0, 0, 1) for y in range(H)] + [(3, y, 100, 200, 255, 2) for y in range(H)]
    cells = _grid(W, H, spec)
    rays = []
    for z in (255 * S - 1, 255 * S, 255 * S + 1, 200 * S, 230 * S):
        for dz in (0, 1, S // 64, -S // 64):
            rays.append(((S // 2, 2 * S + 123, z), (S, S // 3, dz)))
            rays.append(((7 * S + 5, 2 * S + 123, z), (-S, -S // 5, dz)))
    o = np.array([r[0] for r in rays], np.int64)
    d = np.array([r[1] for r in rays], np.int64)
    res = oracle.trace_rays(cells, o, d)
    bad = [k for k in range(len(rays)) if not _same(brute.trace(cells, o[k], d[k]), res, k, W)]
    assert not bad, [rays[k] for k in bad[:5]]
    assert (res["face"] != 255).sum() >= 10
