"""Brute-force checker for the oracle (tiny grids, exact fractions).

TEST INFRASTRUCTURE ONLY, and independent of ``hf_oracle.c``: it does not step
from cell to cell.  For every column of the grid it builds the closed interval
of t over which the ray is inside that column, straight from the definition
(the set of t >= 0 with floor(p(t)/S) equal to the column, kept only when it
has positive length), intersects it with the column's two solid intervals in
z (floor z <= h0 S, slab h1 S <= z <= h2 S: the SOLID predicate of the
paper's Section 3.1), and takes the earliest solid t over all columns, ties
going to the column entered first.
"""

import math
from fractions import Fraction as Fr

S = 65536
INF = math.inf


def _axis_interval(o, d, i):
    """Closure of {t : i S <= o + t d < (i+1) S} as (lo, hi); None if empty."""
    a, b = i * S, (i + 1) * S
    if d == 0:
        return (-INF, INF) if a <= o < b else None
    if d > 0:
        return (Fr(a - o, d), Fr(b - o, d))
    return (Fr(b - o, d), Fr(a - o, d))


def _first_solid(lo, hi, oz, dz, h0, h1, h2):
    """Earliest t in [lo, hi] with z(t) solid in a column, as (t, layer) or None."""
    best = None

    def halfline(level, below):
        # t-set where z(t) <= level (below=True) or z(t) >= level (below=False)
        if dz == 0:
            ok = (oz <= level) if below else (oz >= level)
            return (-INF, INF) if ok else None
        tb = Fr(level - oz, dz)
        rising = dz > 0
        if below == rising:   # z <= level while rising / z >= level while falling
            return (-INF, tb)
        return (tb, INF)

    def meet(*ivs):
        a, b = lo, hi
        for iv in ivs:
            if iv is None:
                return None
            a, b = max(a, iv[0]), min(b, iv[1])
        return a if a <= b else None

    t0 = meet(halfline(h0 * S, True))
    if t0 is not None:
        best = (t0, 0)
    if h1 > h0:
        t1 = meet(halfline(h1 * S, False), halfline(h2 * S, True))
        if t1 is not None and (best is None or t1 < best[0]):
            best = (t1, 1)
    return best


def trace(cells, o, d):
    """(hit_cell, layer, face, depth) of one ray on a small uint32 grid."""
    H, W = cells.shape
    ox, oy, oz = (int(v) for v in o)
    dx, dy, dz = (int(v) for v in d)
    cols = [_axis_interval(ox, dx, i) for i in range(W)]
    rows = [_axis_interval(oy, dy, j) for j in range(H)]
    best = None  # (t, lo, x, y, layer, entry_x)
    for j in range(H):
        ry = rows[j]
        if ry is None:
            continue
        for i in range(W):
            rx = cols[i]
            if rx is None:
                continue
            lo = max(Fr(0), rx[0], ry[0])
            hi = min(rx[1], ry[1])
            if not lo < hi:
                continue
            c = int(cells[j, i])
            h0, h1, h2 = c & 0xFF, (c >> 8) & 0xFF, (c >> 16) & 0xFF
            fs = _first_solid(lo, hi, oz, dz, h0, h1, h2)
            if fs is None:
                continue
            key = (fs[0], lo)
            if best is None or key < (best[0], best[1]):
                best = (fs[0], lo, i, j, fs[1], rx[0] == lo)
    if best is None:
        return 0xFFFFFFFF, 255, 255, INF
    t, lo, i, j, layer, entry_x = best
    if t == lo:
        if lo == 0:
            face = 6
        elif entry_x:
            face = 0 if dx > 0 else 1
        else:
            face = 2 if dy > 0 else 3
    else:
        face = 5 if dz < 0 else 4
    depth = float(t) * math.sqrt(dx * dx + dy * dy + dz * dz) / S
    return j * W + i, layer, face, depth


def pyramid(cells):
    """Min/max pyramid by padding to a power-of-two block and reducing.

    Out-of-grid cells are padded with the identity (max h0 0, min h1 255,
    max top 0); level k is reduced from the padded cells in one step.
    """
    import numpy as np

    c = np.asarray(cells, dtype=np.int64)
    H, W = c.shape
    h0, h1, h2 = c & 0xFF, (c >> 8) & 0xFF, (c >> 16) & 0xFF
    slab = h1 > h0
    a = h0
    b = np.where(slab, h1, 255)
    top = np.where(slab, h2, h0)
    L = 0
    while (1 << L) < max(W, H):
        L += 1
    out = []
    for k in range(1, L + 1):
        n = 1 << k
        hk, wk = -(-H // n), -(-W // n)
        pa = np.zeros((hk * n, wk * n), np.int64)
        pb = np.full((hk * n, wk * n), 255, np.int64)
        pt = np.zeros((hk * n, wk * n), np.int64)
        pa[:H, :W], pb[:H, :W], pt[:H, :W] = a, b, top
        ra = pa.reshape(hk, n, wk, n).max(axis=(1, 3))
        rb = pb.reshape(hk, n, wk, n).min(axis=(1, 3))
        rt = pt.reshape(hk, n, wk, n).max(axis=(1, 3))
        out.append((ra | (rb << 8) | (rt << 16)).astype(np.uint32))
    return out
