"""CPU oracle of the paper's Scattered method (its Section 3: the original
engine's object-order painter recast as a parallel atomic scatter).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's scoring); shares no code
with the CUDA scatter.  Parity unpinned: no -- see tests/test_scatter_pins.py.

The paper gives the shape of the method and leaves its sampling open; this
project's reading (one definition, implemented here and in the CUDA library):

Camera constants (float32, in this order; F, R, U the integer camera vectors,
O the origin in 2^-16 units):
  Of = float32(O) * 2^-16;  cF = 1 / ((Fx*Fx + Fy*Fy) + Fz*Fz), same for cR, cU;
  lr = sqrt(Rx*Rx + Ry*Ry), rh = (Rx/lr, Ry/lr), fh = (-rh_y, rh_x)
  (the ground footprint is aligned with the camera's right vector).
Footprint sample (i, j), 0 <= i < nu, 0 <= j < nv (the "warped footprint"):
  t = (j + 0.5) / nv;  s = s_lo + (s_hi - s_lo) * (t * t)   (quadratic warp:
      samples crowd near s_lo, the camera end of the footprint)
  half = u_min + |s| * k_lat;  u = half * (((i + 0.5) / nu) * 2 - 1)
  (a trapezoid: a pitched camera's view of the ground widens linearly with
  distance from a non-zero width at its near edge)
  x = (Of_x + s*fh_x) + u*rh_x;  y = (Of_y + s*fh_y) + u*rh_y
  the cell (floor x, floor y) (skipped outside the grid) gives the column.
Column walk, m = 0 .. nz-1, tm = m / (nz - 1):
  floor: z = low - low * tm   (mix(low, 0, t)), layer 0
  slab:  z = high + (mid - high) * tm   (mix(high, mid, t)), layer 1, only
         for a cell with a slab.
Projection of P = (x, y, z): v = P - Of; vf = (vx*Fx + vy*Fy) + vz*Fz, same
  for vr (R) and vu (U); a point with vf <= 0 is dropped;
  a = (vr*cR) / (vf*cF), b = (vu*cU) / (vf*cF) (the pixel coordinates of the
  camera model d = F + aR + bU); px = floor((a + w) * 0.5),
  py = floor((h - b) * 0.5); points outside the image are dropped.
Depth = sqrt((vx*vx + vy*vy) + vz*vz) (Euclidean, world units), quantised to
  q = trunc(min(depth * qscale, 2^24 - 1)), qscale = (2^24 - 1) / depth_max;
  packed = q << 8 | (material | layer << 3); the screen keeps the minimum
  (the paper's 32-bit atomicMin of 24 bits of depth and 8 bits of type).
Resolve, per pixel: empty -> miss (hit_cell 0xFFFFFFFF, layer 255, face 255,
  depth +inf, sky colour).  Else depth = float32(q) * dscale,
  dscale = depth_max / (2^24 - 1); the pixel ray d = F + aR + bU (integers),
  dl = sqrt((dx*dx + dy*dy) + dz*dz), k = depth / dl, the point
  (Of_x + dx*k, Of_y + dy*k) gives hit_cell (clamped into the grid); layer
  from the type; face +Z (a point sample has no side); colour = the material's
  albedo lit by the sun on an up-facing surface, no shadow.
All arithmetic is float32, round to nearest, no fused multiply-add.
"""

import numpy as np

f32 = np.float32
QMAX = 16777215  # 2^24 - 1
EMPTY = 0xFFFFFFFF


def camera_constants(cam):
    O = np.asarray(cam["o"], np.int64)
    F = np.asarray(cam["f"], np.int64).astype(f32)
    R = np.asarray(cam["r"], np.int64).astype(f32)
    U = np.asarray(cam["u"], np.int64).astype(f32)
    Of = O.astype(np.int32).astype(f32) * f32(1.0 / 65536.0)

    def inv_sq(V):
        return f32(1.0) / ((V[0] * V[0] + V[1] * V[1]) + V[2] * V[2])

    lr = np.sqrt(R[0] * R[0] + R[1] * R[1])
    rh = (R[0] / lr, R[1] / lr)
    return dict(Of=Of, F=F, R=R, U=U, cF=inv_sq(F), cR=inv_sq(R), cU=inv_sq(U), rh=rh,
                fh=(-rh[1], rh[0]), w=int(cam["w"]), h=int(cam["h"]))


def footprint(k, nu, nv, s_lo, s_hi, k_lat, u_min):
    """Ground positions (x, y) of every footprint sample (float32 [nv, nu])."""
    j = np.arange(nv, dtype=f32)[:, None]
    i = np.arange(nu, dtype=f32)[None, :]
    t = (j + f32(0.5)) / f32(nv)
    s = f32(s_lo) + (f32(s_hi) - f32(s_lo)) * (t * t)
    half = f32(u_min) + np.abs(s) * f32(k_lat)
    u = half * (((i + f32(0.5)) / f32(nu)) * f32(2.0) - f32(1.0))
    x = (k["Of"][0] + s * k["fh"][0]) + u * k["rh"][0]
    y = (k["Of"][1] + s * k["fh"][1]) + u * k["rh"][1]
    return x.astype(f32), y.astype(f32)


def _project(k, x, y, z, depth_max):
    """(pixel index or -1, packed depth without the type) of float32 points."""
    vx, vy, vz = x - k["Of"][0], y - k["Of"][1], z - k["Of"][2]
    F, R, U = k["F"], k["R"], k["U"]
    vf = (vx * F[0] + vy * F[1]) + vz * F[2]
    vr = (vx * R[0] + vy * R[1]) + vz * R[2]
    vu = (vx * U[0] + vy * U[1]) + vz * U[2]
    w, h = k["w"], k["h"]
    with np.errstate(all="ignore"):
        den = vf * k["cF"]
        a = (vr * k["cR"]) / den
        b = (vu * k["cU"]) / den
        pxf = np.floor((a + f32(w)) * f32(0.5))
        pyf = np.floor((f32(h) - b) * f32(0.5))
    ok = (vf > 0) & (pxf >= 0) & (pxf < w) & (pyf >= 0) & (pyf < h)
    d = np.sqrt((vx * vx + vy * vy) + vz * vz)
    qscale = f32(QMAX) / f32(depth_max)
    q = np.minimum(d * qscale, f32(QMAX))
    q = np.where(ok, q, 0).astype(np.uint32)  # truncation of a non-negative float
    pix = np.where(ok, pyf.astype(np.int64) * w + pxf.astype(np.int64), -1)
    return pix, q


def scatter_buffer(cells, cam, nu, nv, nz, s_lo, s_hi, k_lat, u_min, depth_max):
    """The packed screen buffer (uint32 [h*w]) after every point is scattered."""
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    H, W = cells.shape
    k = camera_constants(cam)
    x, y = footprint(k, nu, nv, s_lo, s_hi, k_lat, u_min)
    x, y = x.ravel(), y.ravel()
    cx, cy = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64)
    inside = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
    x, y, cx, cy = x[inside], y[inside], cx[inside], cy[inside]
    c = cells[cy, cx]
    h0 = (c & 0xFF).astype(f32)
    h1 = ((c >> 8) & 0xFF).astype(f32)
    h2 = ((c >> 16) & 0xFF).astype(f32)
    slab = ((c >> 8) & 0xFF) > (c & 0xFF)
    mat = (c >> 24) & 7
    buf = np.full(k["w"] * k["h"], EMPTY, np.uint32)
    for m in range(nz):
        tm = f32(m) / f32(nz - 1)
        for layer, z, sel in ((0, h0 - h0 * tm, np.ones(len(c), bool)),
                              (1, h2 + (h1 - h2) * tm, slab)):
            pix, q = _project(k, x[sel], y[sel], z[sel].astype(f32), depth_max)
            packed = (q << np.uint32(8)) | (mat[sel] | np.uint32(layer << 3)).astype(np.uint32)
            ok = pix >= 0
            np.minimum.at(buf, pix[ok], packed[ok])
    return buf


def resolve(cells, cam, buf, depth_max):
    """Per-pixel outputs from a packed buffer: dict(hit_cell, layer, face,
    depth, material) (material 255 on a miss; `colours` turns it into rgba)."""
    H, W = np.asarray(cells).shape
    k = camera_constants(cam)
    w, h = k["w"], k["h"]
    n = w * h
    hit = buf != EMPTY
    q = (buf >> np.uint32(8)).astype(f32)
    depth = q * (f32(depth_max) / f32(QMAX))
    px = np.arange(n) % w
    py = np.arange(n) // w
    a = 2 * px + 1 - w
    b = h - 1 - 2 * py
    F, R, U = (np.asarray(cam[key], np.int64) for key in ("f", "r", "u"))
    d = [(F[i] + a * R[i] + b * U[i]).astype(np.int32).astype(f32) for i in range(3)]
    dl = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    with np.errstate(all="ignore"):
        kk = depth / dl
        xw = k["Of"][0] + d[0] * kk
        yw = k["Of"][1] + d[1] * kk
        cx = np.clip(np.floor(xw), 0, W - 1).astype(np.int64)
        cy = np.clip(np.floor(yw), 0, H - 1).astype(np.int64)
    typ = buf & np.uint32(0xFF)
    out = dict(
        hit_cell=np.where(hit, (cy * W + cx).astype(np.uint32), np.uint32(EMPTY)).astype(np.uint32),
        layer=np.where(hit, (typ >> 3) & 1, 255).astype(np.uint8),
        face=np.where(hit, 5, 255).astype(np.uint8),
        depth=np.where(hit, depth, np.inf).astype(np.float32),
        material=np.where(hit, typ & 7, 255).astype(np.uint8),
    )
    return out


# the shading of the exact path (the oracle's C source): 8 albedos, ka 0.3, kd 0.7
ALBEDO = np.array([[0.55, 0.50, 0.40], [0.35, 0.55, 0.25], [0.60, 0.60, 0.62], [0.80, 0.72, 0.50],
                   [0.30, 0.30, 0.32], [0.70, 0.35, 0.20], [0.90, 0.90, 0.95], [0.25, 0.40, 0.60]])
SKY = 0xFFEBB487


def colours(material, sun=(321060, -321060, 262144)):
    """rgba of resolved pixels: an up-facing surface lit by the sun, no
    shadow (FP64, rounded half up); sky where material is 255."""
    L = np.asarray(sun, np.float64)
    ndl = max(0.0, L[2] / np.sqrt((L * L).sum()))
    k = 0.3 + 0.7 * ndl
    m = np.where(material == 255, 0, material).astype(np.int64)
    v = np.clip(ALBEDO[m] * k, 0.0, 1.0)
    q = np.floor(255.0 * v + 0.5).astype(np.uint32)
    rgba = np.uint32(0xFF000000) | q[:, 0] | (q[:, 1] << np.uint32(8)) | (q[:, 2] << np.uint32(16))
    return np.where(material == 255, np.uint32(SKY), rgba).astype(np.uint32)


def render(cells, cam, nu, nv, nz, s_lo, s_hi, k_lat, u_min, depth_max):
    buf = scatter_buffer(cells, cam, nu, nv, nz, s_lo, s_hi, k_lat, u_min, depth_max)
    out = resolve(cells, cam, buf, depth_max)
    out["packed"] = buf
    out["rgba"] = colours(out["material"])
    return out
