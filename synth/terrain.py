"""Seeded two-interval terrain grids and crater edits.

Terrain recipe (stands in for the Vangers level of the paper's data section,
which is 2048 x 16384 with a second solid interval on part of the texels):

* h0: 4-octave value noise, base period 128 cells, period halving and weight
  halving per octave (1, 1/2, 1/4, 1/8), lattice values from the counter RNG,
  smoothstep-bilinear interpolation at cell centres, normalised to [0, 1);
  h0 = 20 + floor(100 v + 1/2), so h0 is in [20, 120].
* slab mask: a second noise field (stream 1, base period 64) thresholded at
  its (1 - f) quantile, so a fraction f of cells carries a slab.
* slab heights: h1 = min(255, h0 + U[8, 40]), h2 = min(255, h1 + U[4, 30]).
* material: U[0, 7].
* walls (optional): axis-aligned one-cell ridges of length U[16, 256] with
  h0 = 200 and no slab, flanked on both sides by cells with h0 = 0 and no slab
  (the "0 to 200" jump of an authored cliff).
"""

import hashlib

import numpy as np

from .rng import unit_float, uniform_int

CELL_SLAB_STREAMS = dict(noise=0, mask=1, h1=2, h2=3, mat=4, walls=5)


def _noise_octave_rows(W, y_lo, y_hi, seed, stream, octave, period):
    """One octave of value noise for rows [y_lo, y_hi) of a W-wide grid."""
    xs = np.arange(W)
    cx = xs // period
    fx = ((xs % period) + 0.5) / period
    sx = fx * fx * (3.0 - 2.0 * fx)
    ys = np.arange(y_lo, y_hi)
    cy = ys // period
    fy = ((ys % period) + 0.5) / period
    sy = fy * fy * (3.0 - 2.0 * fy)
    ly0 = int(cy.min())
    ly1 = int(cy.max()) + 2
    lx1 = int(cx.max()) + 2
    iy = np.arange(ly0, ly1, dtype=np.uint64)
    ix = np.arange(0, lx1, dtype=np.uint64)
    idx = (np.uint64(octave) << np.uint64(40)) | (iy[:, None] << np.uint64(20)) | ix[None, :]
    lat = unit_float(seed, stream, idx)
    rowx = lat[:, cx] * (1.0 - sx) + lat[:, cx + 1] * sx
    r = cy - ly0
    return rowx[r] * (1.0 - sy)[:, None] + rowx[r + 1] * sy[:, None]


def value_noise(W, H, seed, stream, base_period, octaves=4, chunk_rows=2048):
    """Value noise in [0, 1) over an H x W grid (float64, row-major)."""
    out = np.empty((H, W), dtype=np.float64)
    weights = [0.5 ** o for o in range(octaves)]
    wsum = sum(weights)
    for y_lo in range(0, H, chunk_rows):
        y_hi = min(H, y_lo + chunk_rows)
        acc = np.zeros((y_hi - y_lo, W), dtype=np.float64)
        for o in range(octaves):
            period = max(1, base_period >> o)
            acc += weights[o] * _noise_octave_rows(W, y_lo, y_hi, seed, stream, o, period)
        out[y_lo:y_hi] = acc / wsum
    return out


def pack_cells(h0, h1, h2, mat):
    """Pack four byte planes into uint32 cell words (byte0 = h0 ... byte3 = mat)."""
    return (np.asarray(h0, np.uint32)
            | (np.asarray(h1, np.uint32) << np.uint32(8))
            | (np.asarray(h2, np.uint32) << np.uint32(16))
            | (np.asarray(mat, np.uint32) << np.uint32(24)))


def unpack_cells(cells):
    """Split uint32 cell words into (h0, h1, h2, mat) int32 planes."""
    c = np.asarray(cells, np.uint32)
    return ((c & 0xFF).astype(np.int32), ((c >> 8) & 0xFF).astype(np.int32),
            ((c >> 16) & 0xFF).astype(np.int32), ((c >> 24) & 0xFF).astype(np.int32))


def _wall_cells(W, H, seed, n_walls):
    """Ridge and flank masks of n_walls axis-aligned one-cell ridges."""
    ridge = np.zeros((H, W), dtype=bool)
    flank = np.zeros((H, W), dtype=bool)
    st = CELL_SLAB_STREAMS["walls"]
    for r in range(n_walls):
        base = 8 * r
        along_y = int(uniform_int(seed, st, base + 0, 0, 1))
        length = int(uniform_int(seed, st, base + 1, 16, 256))
        x0 = int(uniform_int(seed, st, base + 2, 0, W - 1))
        y0 = int(uniform_int(seed, st, base + 3, 0, H - 1))
        if along_y:
            y1 = min(H, y0 + length)
            ridge[y0:y1, x0] = True
            if x0 - 1 >= 0:
                flank[y0:y1, x0 - 1] = True
            if x0 + 1 < W:
                flank[y0:y1, x0 + 1] = True
        else:
            x1 = min(W, x0 + length)
            ridge[y0, x0:x1] = True
            if y0 - 1 >= 0:
                flank[y0 - 1, x0:x1] = True
            if y0 + 1 < H:
                flank[y0 + 1, x0:x1] = True
    return ridge, flank


def make_grid(W, H, seed, slab_frac, n_walls=0):
    """Seeded terrain grid.

    Returns (cells, wall_mask): cells is a uint32 [H, W] array of packed cell
    words; wall_mask marks ridge and flank cells (all False without walls).
    """
    st = CELL_SLAB_STREAMS
    v = value_noise(W, H, seed, st["noise"], 128)
    h0 = (20 + np.floor(100.0 * v + 0.5)).astype(np.int64)
    del v
    N = W * H
    slab = np.zeros((H, W), dtype=bool)
    if slab_frac > 0.0:
        m = value_noise(W, H, seed, st["mask"], 64)
        k = min(N - 1, int(np.floor((1.0 - slab_frac) * N)))
        thr = np.partition(m.ravel(), k)[k]
        slab = m >= thr
        del m
    idx = np.arange(N, dtype=np.uint64).reshape(H, W)
    h1 = np.minimum(255, h0 + uniform_int(seed, st["h1"], idx, 8, 40))
    h2 = np.minimum(255, h1 + uniform_int(seed, st["h2"], idx, 4, 30))
    mat = uniform_int(seed, st["mat"], idx, 0, 7)
    h1 = np.where(slab, h1, 0)
    h2 = np.where(slab, h2, 0)
    wall = np.zeros((H, W), dtype=bool)
    if n_walls:
        ridge, flank = _wall_cells(W, H, seed, n_walls)
        h0 = np.where(flank, 0, h0)
        h1 = np.where(flank, 0, h1)
        h2 = np.where(flank, 0, h2)
        h0 = np.where(ridge, 200, h0)
        h1 = np.where(ridge, 0, h1)
        h2 = np.where(ridge, 0, h2)
        wall = ridge | flank
    return pack_cells(h0, h1, h2, mat), wall


def grid_hash(cells):
    """64-bit BLAKE2b digest (hex) of the grid's little-endian bytes."""
    c = np.ascontiguousarray(np.asarray(cells, dtype="<u4"))
    return hashlib.blake2b(c.tobytes(), digest_size=8).hexdigest()


def crater_edit(cells, cx, cy, size=64, depth=40, r_full=32, r_slab=20):
    """Crater edit centred on cell (cx, cy), as a rectangle of new cells.

    Inside the size x size rectangle [cx - size/2, cx + size/2) (clipped to the
    grid), with r2 = dx*dx + dy*dy from the centre cell: for r2 < r_full**2
    the floor is lowered by floor(depth * (r_full**2 - r2) / r_full**2)
    (clamped at 0), and for r2 < r_slab**2 the upper slab is removed.
    Outside the slab radius the slab stays valid because h0 only decreases.

    Returns (x0, y0, block) with block a uint32 [h, w] array; the caller
    writes it into its copy of the grid.
    """
    H, W = cells.shape
    half = size // 2
    x0 = max(0, cx - half)
    y0 = max(0, cy - half)
    x1 = min(W, cx + half)
    y1 = min(H, cy + half)
    block = np.array(cells[y0:y1, x0:x1], dtype=np.uint32)
    h0, h1, h2, mat = unpack_cells(block)
    yy, xx = np.mgrid[y0:y1, x0:x1]
    r2 = (xx - cx) ** 2 + (yy - cy) ** 2
    rf2 = r_full * r_full
    drop = np.where(r2 < rf2, (depth * (rf2 - r2)) // rf2, 0)
    h0 = np.maximum(0, h0 - drop)
    kill = r2 < r_slab * r_slab
    h1 = np.where(kill, 0, h1)
    h2 = np.where(kill, 0, h2)
    return x0, y0, pack_cells(h0, h1, h2, mat)
