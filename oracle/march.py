"""CPU oracle of the paper's fixed-step height-field ray march (Section 3.1).

TEST INFRASTRUCTURE ONLY (tests, and the benchmark's scoring of the marcher);
shares no code with the CUDA marcher.

What it computes, per pixel ray p(t) = o + t d (world units: o = origin / 2^16,
d = integer direction / 2^16, so t is the same parameter as the exact cast's):
  * the segment [0, t_end] is clipped at the far distance (t_far = far / |d|)
    and, for a descending ray, at z = 0 (t_z = -o_z / d_z);
  * `steps` samples at t_i = i * (t_end / (steps + 1)), i = 1..steps, spaced
    uniformly over the clipped segment (as the text describes; the listing
    moves the lower bound inside its loop, which would space them
    geometrically and never reach the far part, so the text is taken);
  * the first sample whose point is SOLID stops the search: z <= low, or
    mid <= z <= high, for the cell containing the point's x, y (floor; no
    solid outside the grid);
  * four bisections of [t_prev, t_hit] keep the solid end;
  * a ray with no solid sample misses (no hit is made at the ground plane).
Output: hit cell index (or 0xFFFFFFFF), layer of the solid interval at the hit
point (0 floor, 1 slab, 255 miss), depth = t_hit * |d|.

Every operation is float32 with round-to-nearest and no fused multiply-add,
in the order written here, so a float32 kernel that performs the same
operations in the same order reproduces it bit for bit.
"""

import numpy as np

f32 = np.float32
INV_S = f32(1.0 / 65536.0)


def _solid(cells, x, y, z):
    """SOLID at float32 points: (solid mask, cell index, layer)."""
    H, W = cells.shape
    cx = np.floor(x).astype(np.int64)
    cy = np.floor(y).astype(np.int64)
    inside = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
    c = np.zeros(x.shape, np.uint32)
    c[inside] = cells[cy[inside], cx[inside]]
    h0 = (c & 0xFF).astype(np.float32)
    h1 = ((c >> 8) & 0xFF).astype(np.float32)
    h2 = ((c >> 16) & 0xFF).astype(np.float32)
    slab = ((c >> 8) & 0xFF) > (c & 0xFF)
    floor_ = z <= h0
    upper = slab & (z >= h1) & (z <= h2)
    solid = inside & (floor_ | upper)
    idx = np.where(inside, cy * W + cx, -1)
    layer = np.where(floor_, 0, 1)
    return solid, idx, layer


def march(cells, origin, dirs, steps=128, far=600.0, bisections=4):
    """March rays from origins (int64 [3] shared, or [n, 3]; 2^-16 units) along
    integer directions dirs (int64 [n, 3]).  Returns dict(hit_cell, layer, depth)."""
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    dirs = np.asarray(dirs, np.int64).reshape(-1, 3)
    n = dirs.shape[0]
    org = np.broadcast_to(np.asarray(origin, np.int64).reshape(-1, 3), (n, 3))
    o = [(org[:, k].astype(np.float32) * INV_S).astype(f32) for k in range(3)]
    d = [(dirs[:, k].astype(np.float32) * INV_S).astype(np.float32) for k in range(3)]
    sq = (d[0] * d[0]).astype(f32)
    sq = (sq + (d[1] * d[1]).astype(f32)).astype(f32)
    sq = (sq + (d[2] * d[2]).astype(f32)).astype(f32)
    length = np.sqrt(sq).astype(f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        t_end = (f32(far) / length).astype(f32)
        t_z = ((-o[2]).astype(f32) / d[2]).astype(f32)
    down = d[2] < 0
    t_end = np.where(down & (t_z < t_end), t_z, t_end).astype(f32)
    dt = (t_end / f32(steps + 1)).astype(f32)

    def point(t):
        return [(o[k] + (t * d[k]).astype(f32)).astype(f32) for k in range(3)]

    found = np.zeros(n, bool)
    a = np.zeros(n, f32)
    b = np.zeros(n, f32)
    for i in range(1, steps + 1):
        t = (f32(i) * dt).astype(f32)
        p = point(t)
        s, _, _ = _solid(cells, *p)
        new = s & ~found
        b = np.where(new, t, b)
        a = np.where(new, (f32(i - 1) * dt).astype(f32), a)
        found |= s
    for _ in range(bisections):
        m = ((a + b).astype(f32) * f32(0.5)).astype(f32)
        s, _, _ = _solid(cells, *point(m))
        b = np.where(found & s, m, b)
        a = np.where(found & ~s, m, a)
    p = point(b)
    _, idx, layer = _solid(cells, *p)
    depth = (b * length).astype(f32)
    hit_cell = np.where(found, idx, 0xFFFFFFFF).astype(np.uint32)
    return dict(hit_cell=hit_cell, layer=np.where(found, layer, 255).astype(np.uint8),
                depth=np.where(found, depth, np.inf).astype(np.float32))


def march_camera(cells, cam, steps=128, far=600.0, bisections=4):
    """March every pixel of a camera record (same ray model as the exact cast)."""
    from . import ray_dirs

    return march(cells, np.array(cam["o"], np.int64), ray_dirs(cam), steps, far, bisections)
