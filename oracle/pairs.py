"""Decoder of the paired-texel world encoding -- TEST INFRASTRUCTURE ONLY (the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU legs call it; the
product never imports it).

The paper's data section describes Vangers' height map: a texel holds one
altitude, except in double-level regions, where a *pair* of texels (even x,
odd x) describes one column with three altitudes -- the even texel stores the
floor top ``low``, the odd texel the slab top ``high``, and the cave ceiling
``mid`` is derived from delta bits carried by both.  The paper does not give
the bit layout; this project's reading (one definition, implemented twice:
here and in the CUDA library) is:

  texel  = uint16, little-endian: low byte = altitude v, high byte = meta m
  m bit 7      D, the pair is double-level (equal on both texels of a pair)
  m bits 6..3  a delta nibble
  m bits 2..0  material

  single-level pair (D = 0): each texel is its own cell,
      h0 = v, no slab (h1 = h2 = 0), material = m & 7; both nibbles are 0
  double-level pair (D = 1): both cells of the pair have
      h0 = low = v(even), h2 = high = v(odd),
      h1 = mid = high - (16 * nibble(even) + nibble(odd)),
      and the material of their own texel; valid only when low < mid <= high
      (a slab above the floor, possibly of zero thickness, mid = high)

A grid in this encoding has an even width.  Decoding gives the ordinary
cell words (byte0 h0, byte1 h1, byte2 h2, byte3 material) that the rest of
the oracle renders.  Parity unpinned: no -- the decoder is pinned by
hand-derived texel pairs (tests/golden/pair_codec.json) and by round trips.
"""

import numpy as np


def _split(texels):
    t = np.asarray(texels, dtype=np.uint16)
    if t.ndim != 2 or t.shape[1] % 2:
        raise ValueError("paired texels need a 2-D array of even width")
    v = (t & 0xFF).astype(np.int64)
    m = (t >> 8).astype(np.int64)
    return v, m


def validate_loop(texels):
    """Returns (ok, first bad texel index in row-major order or None); one
    pair at a time (small grids)."""
    v, m = _split(texels)
    H, W = v.shape
    for y in range(H):
        for k in range(0, W, 2):
            ve, vo, me, mo = v[y, k], v[y, k + 1], m[y, k], m[y, k + 1]
            de, do = me >> 7, mo >> 7
            if de != do:
                return False, y * W + k
            if de == 0:
                if (me >> 3) & 15 or (mo >> 3) & 15:
                    return False, y * W + k
                continue
            delta = 16 * ((me >> 3) & 15) + ((mo >> 3) & 15)
            mid = vo - delta
            if not (ve < mid <= vo):
                return False, y * W + k
    return True, None


def decode_loop(texels):
    """Cell words (uint32, same shape) of a valid paired-texel grid, one cell
    at a time straight from the definition (small grids)."""
    ok, bad = validate_loop(texels)
    if not ok:
        raise ValueError("invalid paired texel at index %d" % bad)
    v, m = _split(texels)
    H, W = v.shape
    out = np.zeros((H, W), dtype=np.uint32)
    for y in range(H):
        for x in range(W):
            e, o = x - (x % 2), x - (x % 2) + 1
            mat = int(m[y, x]) & 7
            if m[y, e] >> 7:
                low, high = int(v[y, e]), int(v[y, o])
                mid = high - (16 * ((int(m[y, e]) >> 3) & 15) + ((int(m[y, o]) >> 3) & 15))
                h0, h1, h2 = low, mid, high
            else:
                h0, h1, h2 = int(v[y, x]), 0, 0
            out[y, x] = h0 | (h1 << 8) | (h2 << 16) | (mat << 24)
    return out


def validate(texels):
    """validate_loop over whole arrays (any size)."""
    v, m = _split(texels)
    H, W = v.shape
    ve, vo, me, mo = v[:, 0::2], v[:, 1::2], m[:, 0::2], m[:, 1::2]
    de, do = me >> 7, mo >> 7
    ne, no = (me >> 3) & 15, (mo >> 3) & 15
    mid = vo - (16 * ne + no)
    bad = (de != do) | ((de == 0) & ((ne != 0) | (no != 0))) | ((de == 1) & ~((ve < mid) & (mid <= vo)))
    if not bad.any():
        return True, None
    y, k = np.argwhere(bad)[0]
    return False, int(y) * W + 2 * int(k)


def decode(texels):
    """decode_loop over whole arrays (any size)."""
    ok, bad = validate(texels)
    if not ok:
        raise ValueError("invalid paired texel at index %d" % bad)
    v, m = _split(texels)
    ve, vo, me, mo = v[:, 0::2], v[:, 1::2], m[:, 0::2], m[:, 1::2]
    dual = (me >> 7) == 1
    mid = vo - (16 * ((me >> 3) & 15) + ((mo >> 3) & 15))
    h0 = np.empty_like(v)
    h1 = np.zeros_like(v)
    h2 = np.zeros_like(v)
    h0[:, 0::2] = ve
    h0[:, 1::2] = np.where(dual, ve, vo)
    for par in (0, 1):
        h1[:, par::2] = np.where(dual, mid, 0)
        h2[:, par::2] = np.where(dual, vo, 0)
    mat = m & 7
    return (h0 | (h1 << 8) | (h2 << 16) | (mat << 24)).astype(np.uint32)
