"""Seeded inputs in the paired-texel world encoding (2 bytes per texel).

Texel = uint16: low byte altitude, high byte meta (bit 7 = the pair is
double-level, bits 6..3 = delta nibble, bits 2..0 = material).  In a
double-level pair (even x, odd x) both cells share one column: the even texel
holds the floor top, the odd texel the slab top, and the slab underside is the
slab top minus 16 * nibble(even) + nibble(odd).

`pairify` turns an ordinary cell grid into one this encoding can hold (a
double-level pair shares its three heights), and `encode_pairs` packs such a
grid into texels.  Neither decodes: decoding is the method's, implemented by
the CUDA library and, separately, by the oracle.
"""

import numpy as np

from .terrain import pack_cells, unpack_cells


def pairify(cells):
    """A copy of `cells` (even width) in which every pair (2k, 2k+1) of a row
    either has no slab in either cell, or both cells carry the same
    (h0, h1, h2): the slab cell's heights (the even cell's when both have one).
    Materials stay per cell."""
    c = np.asarray(cells, dtype=np.uint32)
    if c.ndim != 2 or c.shape[1] % 2:
        raise ValueError("pairify needs a 2-D grid of even width")
    h0, h1, h2, mat = (a.astype(np.int64) for a in unpack_cells(c))
    slab = h1 > h0
    se, so = slab[:, 0::2], slab[:, 1::2]
    src = np.where(se, 0, 1)  # which cell of the pair gives the heights
    any_slab = se | so
    out = [h0.copy(), h1.copy(), h2.copy()]
    for a, o in zip((h0, h1, h2), out):
        pick = np.where(src == 0, a[:, 0::2], a[:, 1::2])
        o[:, 0::2] = np.where(any_slab, pick, a[:, 0::2])
        o[:, 1::2] = np.where(any_slab, pick, a[:, 1::2])
    return pack_cells(out[0], out[1], out[2], mat)


def encode_pairs(cells):
    """uint16 texels of a grid that `pairify` leaves unchanged.  Raises
    ValueError for a grid the encoding cannot hold."""
    c = np.asarray(cells, dtype=np.uint32)
    if c.ndim != 2 or c.shape[1] % 2:
        raise ValueError("paired texels need an even width")
    h0, h1, h2, mat = (a.astype(np.int64) for a in unpack_cells(c))
    slab = h1 > h0
    se, so = slab[:, 0::2], slab[:, 1::2]
    same = ((h0[:, 0::2] == h0[:, 1::2]) & (h1[:, 0::2] == h1[:, 1::2])
            & (h2[:, 0::2] == h2[:, 1::2]))
    if ((se != so) | (se & ~same)).any():
        raise ValueError("grid is not pair-representable (use pairify)")
    delta = np.where(se, h2[:, 0::2] - h1[:, 0::2], 0)  # 0..254
    v = h0.copy()
    v[:, 1::2] = np.where(so, h2[:, 1::2], h0[:, 1::2])
    meta = mat.copy()
    meta[:, 0::2] |= np.where(se, 0x80 | ((delta >> 4) << 3), 0)
    meta[:, 1::2] |= np.where(so, 0x80 | ((delta & 15) << 3), 0)
    return (v | (meta << 8)).astype(np.uint16)
