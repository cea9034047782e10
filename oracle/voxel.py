"""CPU oracle of the paper's voxel-accelerated ray march, RayVoxel (its
Section 3) -- TEST INFRASTRUCTURE ONLY; shares no code with the CUDA version.

The paper's shape: a conservative occupancy pyramid (finest level one bit per
voxel, each higher level the union of its eight children) and a hierarchical
DDA that advances an empty cell straight to its exit plane, descends into an
occupied one, and at the leaf level tests the original height data with fixed
sampling.  It skips only known-empty space, and like the fixed-step march it
can miss a feature thinner than its leaf sampling.  This project's reading
(one definition, implemented here and in the CUDA library):

Occupancy.  Voxel (i, j, k) of level 0 covers cells x in [i vx, (i+1) vx),
y in [j vy, (j+1) vy) (those inside the grid) and heights z in the closed
range [k vz, (k+1) vz]; it is occupied when some cell there is solid at some
such z: z0 <= h0, or a slab with h1 <= z1 and z0 <= h2.  nz0 = ceil(256 / vz)
layers cover every height.  Level l + 1 voxel (i, j, k) = OR of the level-l
voxels (2i + a, 2j + b, 2k + c), a, b, c in {0, 1} (missing ones empty).

Traversal, per pixel ray (float32; o = origin / 2^16, d = integer direction /
2^16, so t is the exact cast's parameter):
  box: the voxel grid [0, nx0 vx] x [0, ny0 vy] x [0, nz0 vz]; slab entry and
    exit t0, t1 (t0 >= 0; t1 <= far / |d|); t0 >= t1 -> miss.
  start at level `top` at p(t0), index floor(p / size) clamped into the level.
  repeat at most `outer` times:
    t_out = the least exit time of the current voxel over the axes
      (axis a: ((i_a + [d_a > 0]) * size_a - o_a) * (1 / d_a); +inf if d_a = 0)
    (a voxel past the level's end, a missing child of the last parent of an
    odd count, is empty)
    occupied and level > 0: go one level down, to the child the ray is in
      just after t: on the axis it last stepped across, the first child along
      its direction; on the other axes (all of them before the first step)
      the child holding p(t) (floor(p / size) clamped into the two children)
    occupied leaf: `inner` samples at t + (min(t_out, t1) - t) (k + 0.5) / inner;
      the first SOLID one (the cell holding the point, z <= h0 -> floor, a slab
      with h1 <= z <= h2 -> slab) is the hit, depth = t |d|
    t_out >= t1 -> miss.  Else step the first axis (x, y, z order) whose exit
      time is t_out by the sign of d; t = t_out; outside the level -> miss;
      when the crossed boundary is a boundary of the parent (the new index is
      even going up, odd going down) and level < top: go one level up.
  the budget exhausted -> miss.
All arithmetic float32, round to nearest, no fused multiply-add, in this order.
"""

import numpy as np

f32 = np.float32
INF = f32(np.inf)


# --------------------------------------------------------------- occupancy

def level0(cells, vx, vy, vz):
    """Dense bool [nz0, ny0, nx0] level-0 occupancy, on whole arrays: a cell's
    floor fills layers 0 .. floor(h0 / vz) (z0 = k vz <= h0), its slab layers
    ceil(h1 / vz) - 1 .. floor(h2 / vz) (h1 <= (k+1) vz and k vz <= h2); a
    voxel column takes the union over its cells (the floor part as a maximum,
    the slab part through a difference array over the layers)."""
    c = np.asarray(cells, np.uint32)
    H, W = c.shape
    h0 = (c & 0xFF).astype(np.int64)
    h1 = ((c >> 8) & 0xFF).astype(np.int64)
    h2 = ((c >> 16) & 0xFF).astype(np.int64)
    slab = h1 > h0
    nx0, ny0, nz0 = -(-W // vx), -(-H // vy), -(-256 // vz)
    ys, xs = np.mgrid[0:H, 0:W]
    col = (ys // vy) * nx0 + (xs // vx)  # voxel column of each cell
    kf = np.full(ny0 * nx0, -1, np.int64)
    np.maximum.at(kf, col.ravel(), np.minimum(h0 // vz, nz0 - 1).ravel())
    diff = np.zeros((ny0 * nx0, nz0 + 1), np.int64)
    ka = np.maximum(0, -(-h1 // vz) - 1)[slab]
    kb = np.minimum(h2 // vz, nz0 - 1)[slab]
    cs = col[slab]
    keep = ka <= kb
    np.add.at(diff, (cs[keep], ka[keep]), 1)
    np.add.at(diff, (cs[keep], kb[keep] + 1), -1)
    slab_occ = np.cumsum(diff[:, :nz0], axis=1) > 0
    occ = slab_occ | (np.arange(nz0)[None, :] <= kf[:, None])
    return np.ascontiguousarray(occ.T.reshape(nz0, ny0, nx0))


def level0_loop(cells, vx, vy, vz):
    """level0 one voxel and one cell at a time (tiny grids; pins level0)."""
    c = np.asarray(cells, np.uint32)
    H, W = c.shape
    nx0, ny0, nz0 = -(-W // vx), -(-H // vy), -(-256 // vz)
    occ = np.zeros((nz0, ny0, nx0), bool)
    for k in range(nz0):
        for j in range(ny0):
            for i in range(nx0):
                z0, z1 = k * vz, (k + 1) * vz
                for y in range(j * vy, min((j + 1) * vy, H)):
                    for x in range(i * vx, min((i + 1) * vx, W)):
                        w = int(c[y, x])
                        a0, a1, a2 = w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFF
                        if z0 <= a0 or (a1 > a0 and a1 <= z1 and z0 <= a2):
                            occ[k, j, i] = True
    return occ


def pyramid(cells, vx, vy, vz, levels):
    """[level 0, ..., level levels-1] dense occupancy arrays."""
    out = [level0(cells, vx, vy, vz)]
    for _ in range(1, levels):
        a = out[-1]
        nz, ny, nx = a.shape
        p = np.zeros((nz + nz % 2, ny + ny % 2, nx + nx % 2), bool)
        p[:nz, :ny, :nx] = a
        out.append(p.reshape(p.shape[0] // 2, 2, p.shape[1] // 2, 2, p.shape[2] // 2, 2)
                   .any(axis=(1, 3, 5)))
    return out


def morton3(x, y, z):
    """Bit index of (x, y, z) in an 8 x 8 x 8 tile: bits interleaved x, y, z
    from the lowest."""
    m = 0
    for b in range(3):
        m |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return m


def pack(level):
    """uint32 words of one level in Morton-coded 8^3 tiles: tile (tx, ty, tz)
    at (tz * TY + ty) * TX + tx, 16 words per tile, bit morton3(x&7, y&7, z&7)."""
    nz, ny, nx = level.shape
    TX, TY, TZ = -(-nx // 8), -(-ny // 8), -(-nz // 8)
    words = np.zeros(TX * TY * TZ * 16, np.uint32)
    z, y, x = (a.astype(np.int64) for a in np.nonzero(level))
    tile = ((z >> 3) * TY + (y >> 3)) * TX + (x >> 3)
    m = np.zeros(len(x), np.int64)
    for b in range(3):  # morton3, on whole arrays
        m |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    np.bitwise_or.at(words, tile * 16 + (m >> 5), (np.uint32(1) << (m & 31).astype(np.uint32)))
    return words


def pack_loop(level):
    """pack, one voxel at a time with morton3 (small levels; pins pack)."""
    nz, ny, nx = level.shape
    TX, TY, TZ = -(-nx // 8), -(-ny // 8), -(-nz // 8)
    words = np.zeros(TX * TY * TZ * 16, np.uint32)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if level[z, y, x]:
                    m = morton3(x & 7, y & 7, z & 7)
                    t = ((z >> 3) * TY + (y >> 3)) * TX + (x >> 3)
                    words[t * 16 + (m >> 5)] |= np.uint32(1 << (m & 31))
    return words


# --------------------------------------------------------------- traversal

def _solid(cells, x, y, z):
    """SOLID at float32 points: (mask, cell index, layer) -- as the march."""
    H, W = cells.shape
    cx = np.floor(x).astype(np.int64)
    cy = np.floor(y).astype(np.int64)
    inside = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
    c = np.zeros(np.shape(x), np.uint32)
    c[inside] = cells[cy[inside], cx[inside]]
    h0 = (c & 0xFF).astype(f32)
    h1 = ((c >> 8) & 0xFF).astype(f32)
    h2 = ((c >> 16) & 0xFF).astype(f32)
    slab = ((c >> 8) & 0xFF) > (c & 0xFF)
    fl = z <= h0
    up = slab & (z >= h1) & (z <= h2)
    return inside & (fl | up), np.where(inside, cy * W + cx, -1), np.where(fl, 0, 1)


class Grid:
    """The occupancy pyramid and its dimensions, as the traversal reads it."""

    def __init__(self, cells, vx, vy, vz, levels):
        self.cells = np.ascontiguousarray(cells, np.uint32)
        self.v = (vx, vy, vz)
        self.levels = pyramid(cells, vx, vy, vz, levels)
        self.dims = [lv.shape[::-1] for lv in self.levels]  # (nx, ny, nz)
        self.flat = np.concatenate([lv.ravel() for lv in self.levels])
        self.off = np.cumsum([0] + [lv.size for lv in self.levels])[:-1]
        self.top = levels - 1

    def occupied(self, l, ix, iy, iz):
        """A voxel past the level's end (a missing child of the last parent
        of an odd count) is empty."""
        nx = np.array([d[0] for d in self.dims])[l]
        ny = np.array([d[1] for d in self.dims])[l]
        nz = np.array([d[2] for d in self.dims])[l]
        inside = (ix < nx) & (iy < ny) & (iz < nz)
        k = self.off[l] + (np.minimum(iz, nz - 1) * ny + np.minimum(iy, ny - 1)) * nx + np.minimum(ix, nx - 1)
        return inside & self.flat[k]


def _setup(g, origin, dirs, far):
    """float32 o, d, 1/d and the box entry/exit t0, t1 per ray."""
    org = np.broadcast_to(np.asarray(origin, np.int64).reshape(-1, 3), dirs.shape)
    s = f32(1.0 / 65536.0)
    o = [org[:, a].astype(np.int32).astype(f32) * s for a in range(3)]
    d = [dirs[:, a].astype(np.int32).astype(f32) * s for a in range(3)]
    n0 = g.dims[0]
    box = [f32(n0[a] * g.v[a]) for a in range(3)]
    dl = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    with np.errstate(all="ignore"):
        t0 = np.zeros(len(dirs), f32)
        t1 = f32(far) / dl
        inv = []
        for a in range(3):
            nz_ = d[a] != 0
            ia = np.where(nz_, f32(1.0) / np.where(nz_, d[a], f32(1.0)), f32(0.0)).astype(f32)
            inv.append(ia)
            ta = (f32(0.0) - o[a]) * ia
            tb = (box[a] - o[a]) * ia
            lo = np.where(nz_, np.minimum(ta, tb), -INF)
            hi = np.where(nz_, np.maximum(ta, tb), INF)
            outside = ~nz_ & ((o[a] < 0) | (o[a] > box[a]))
            t0 = np.maximum(t0, lo)
            t1 = np.where(outside, f32(-1.0), np.minimum(t1, hi))
    return o, d, inv, dl, t0.astype(f32), t1.astype(f32)


def trace(g, origin, dirs, far=600.0, outer=4096, inner=4):
    """Vectorised traversal of rays (integer dirs [n, 3], origin [3] or [n, 3]).
    Returns dict(hit_cell, layer, depth, steps)."""
    dirs = np.asarray(dirs, np.int64).reshape(-1, 3)
    n = len(dirs)
    o, d, inv, dl, t0, t1 = _setup(g, origin, dirs, far)
    top = g.top
    sz = lambda l, a: np.array([g.v[a] << k for k in range(top + 1)], np.float32)[l]
    nn = lambda l, a: np.array([g.dims[k][a] for k in range(top + 1)], np.int64)[l]
    active = t0 < t1
    t = t0.copy()
    lvl = np.full(n, top, np.int64)
    ent = np.full(n, -1, np.int64)  # axis of the last step
    idx = []
    with np.errstate(all="ignore"):
        for a in range(3):
            p = o[a] + d[a] * t
            idx.append(np.clip(np.floor(p / sz(lvl, a)), 0, nn(lvl, a) - 1).astype(np.int64))
    hit_cell = np.full(n, 0xFFFFFFFF, np.uint32)
    layer = np.full(n, 255, np.uint8)
    depth = np.full(n, np.inf, np.float32)
    steps = np.zeros(n, np.int64)
    pos = lambda a, tt, sel: o[a][sel] + d[a][sel] * tt
    for _ in range(outer):
        if not active.any():
            break
        r = np.nonzero(active)[0]
        steps[r] += 1
        l = lvl[r]
        tout = []
        for a in range(3):
            bnd = ((idx[a][r] + (d[a][r] > 0)) * (np.int64(g.v[a]) << l)).astype(f32)
            ta = np.where(d[a][r] != 0, (bnd - o[a][r]) * inv[a][r], INF).astype(f32)
            tout.append(ta)
        t_out = np.minimum(np.minimum(tout[0], tout[1]), tout[2])
        occ = g.occupied(l, idx[0][r], idx[1][r], idx[2][r])
        # descend
        dn = occ & (l > 0)
        if dn.any():
            rd = r[dn]
            lvl[rd] -= 1
            for a in range(3):
                p = pos(a, t[rd], rd)
                c = np.floor(p / sz(lvl[rd], a)).astype(np.int64)
                c = np.clip(c, 2 * idx[a][rd], 2 * idx[a][rd] + 1)
                first = 2 * idx[a][rd] + (d[a][rd] < 0)
                idx[a][rd] = np.where(ent[rd] == a, first, c)
        # sample an occupied leaf
        lf = occ & (l == 0)
        found = np.zeros(len(r), bool)
        if lf.any():
            rl = r[lf]
            th = np.minimum(t_out[lf], t1[rl])
            span = th - t[rl]
            got = np.zeros(len(rl), bool)
            for k in range(inner):
                frac = (f32(k) + f32(0.5)) / f32(inner)
                ts = t[rl] + span * frac
                sol, cell, lay = _solid(g.cells, pos(0, ts, rl), pos(1, ts, rl), pos(2, ts, rl))
                new = sol & ~got
                hit_cell[rl[new]] = cell[new].astype(np.uint32)
                layer[rl[new]] = lay[new]
                depth[rl[new]] = ts[new] * dl[rl[new]]
                got |= sol
            found[np.nonzero(lf)[0][got]] = True
            active[rl[got]] = False
        # advance (rays that neither descended nor hit)
        adv = ~dn & ~found
        ra = r[adv]
        ta_ = t_out[adv]
        stop = ta_ >= t1[ra]
        active[ra[stop]] = False
        ra, ta_ = ra[~stop], ta_[~stop]
        tx, ty, tz = tout[0][adv][~stop], tout[1][adv][~stop], tout[2][adv][~stop]
        ax = np.where(tx == ta_, 0, np.where(ty == ta_, 1, 2))
        t[ra] = ta_
        ent[ra] = ax
        out = np.zeros(len(ra), bool)
        up = np.zeros(len(ra), bool)
        for a in range(3):
            m = ax == a
            sgn = np.where(d[a][ra[m]] > 0, 1, -1)
            idx[a][ra[m]] += sgn
            ia = idx[a][ra[m]]
            out[m] = (ia < 0) | (ia >= nn(lvl[ra[m]], a))
            up[m] = np.where(sgn > 0, ia % 2 == 0, ia % 2 == 1)
        active[ra[out]] = False
        asc = up & ~out & (lvl[ra] < top)
        rs = ra[asc]
        lvl[rs] += 1
        for a in range(3):
            idx[a][rs] >>= 1
    return dict(hit_cell=hit_cell, layer=layer, depth=depth, steps=steps)


def trace_one(g, origin, direction, far=600.0, outer=4096, inner=4, visits=None):
    """The same traversal for one ray, one step at a time (the plain form the
    vectorised `trace` must equal).  `visits` (a list) receives every
    (level, ix, iy, iz, occupied) the ray inspects."""
    o, d, inv, dl, t0, t1 = _setup(g, origin, np.asarray(direction, np.int64).reshape(1, 3), far)
    o, d, inv = [x[0] for x in o], [x[0] for x in d], [x[0] for x in inv]
    dl, t0, t1 = dl[0], t0[0], t1[0]
    if not t0 < t1:
        return None
    top = g.top
    l, t, ent = top, t0, -1
    size = lambda l, a: f32(g.v[a] << l)
    idx = [int(min(max(np.floor((o[a] + d[a] * t) / size(l, a)), 0), g.dims[l][a] - 1)) for a in range(3)]
    for _ in range(outer):
        tout = []
        for a in range(3):
            if d[a] == 0:
                tout.append(INF)
                continue
            b = f32((idx[a] + (1 if d[a] > 0 else 0)) * (g.v[a] << l))
            tout.append((b - o[a]) * inv[a])
        t_out = min(min(tout[0], tout[1]), tout[2])
        inside = idx[0] < g.dims[l][0] and idx[1] < g.dims[l][1] and idx[2] < g.dims[l][2]
        occ = inside and bool(g.levels[l][idx[2], idx[1], idx[0]])
        if visits is not None:
            visits.append((l, idx[0], idx[1], idx[2], occ, float(t)))
        if occ and l > 0:
            l -= 1
            idx = [2 * idx[a] + (1 if d[a] < 0 else 0) if a == ent else
                   int(min(max(np.floor((o[a] + d[a] * t) / size(l, a)), 2 * idx[a]), 2 * idx[a] + 1))
                   for a in range(3)]
            continue
        if occ:
            th = min(t_out, t1)
            for k in range(inner):
                ts = t + (th - t) * ((f32(k) + f32(0.5)) / f32(inner))
                p = [np.array([o[a] + d[a] * ts], f32) for a in range(3)]
                sol, cell, lay = _solid(g.cells, *p)
                if sol[0]:
                    return int(cell[0]), int(lay[0]), f32(ts * dl)
        if t_out >= t1:
            return None
        a = 0 if tout[0] == t_out else (1 if tout[1] == t_out else 2)
        s = 1 if d[a] > 0 else -1
        idx[a] += s
        t, ent = t_out, a
        if idx[a] < 0 or idx[a] >= g.dims[l][a]:
            return None
        if l < top and (idx[a] % 2 == 0 if s > 0 else idx[a] % 2 == 1):
            l += 1
            idx = [i >> 1 for i in idx]
    return None
