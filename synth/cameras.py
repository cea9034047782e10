"""Seeded camera poses and their integer camera records.

Camera record (the integer form every ray caster here consumes):
  origin  int64[3]  position in units of 2**-16 world units (1 world unit =
                    one cell width = one height step)
  fwd     int32[3]  F
  right   int32[3]  R
  up      int32[3]  U
  w, h    uint32    image size in pixels
Pixel (px, py), py = 0 at the top, looks along
  d = F + (2 px + 1 - w) R + (h - 1 - 2 py) U.

A pose (x, y, z, yaw, pitch, hfov) is quantised once, in float64:
  forward = (sin yaw cos pitch, cos yaw cos pitch, sin pitch)   (yaw 0 = +y,
  yaw 90 = +x, pitch < 0 looks down), right = (cos yaw, -sin yaw, 0),
  up = right x forward; the focal length is f = (w/2) / tan(hfov/2) pixels
  (fixed in pixels, never scaled by the image height, the first of the two
  reference-camera mistakes recorded in the paper's evaluation section);
  F = rnd(2**19 forward), R = rnd(2**18 / f * right), U = rnd(2**18 / f * up),
  origin = rnd(2**16 (x, y, z)), with rnd rounding half away from zero.
"""

import math

import numpy as np

from .rng import unit_float, uniform_int
from .terrain import make_grid, unpack_cells

S = 65536

CAMERA_DTYPE = np.dtype(
    [("o", "<i8", (3,)), ("f", "<i4", (3,)), ("r", "<i4", (3,)),
     ("u", "<i4", (3,)), ("w", "<u4"), ("h", "<u4")],
    align=True,
)


def _rnd(v):
    return int(math.copysign(math.floor(abs(v) + 0.5), v))


def pose_to_camera(x, y, z, yaw_deg, pitch_deg, hfov_deg, w, h):
    """Quantise a pose into an integer camera record (tuple form)."""
    yaw = math.radians(yaw_deg)
    pitch = math.radians(pitch_deg)
    sy, cy = math.sin(yaw), math.cos(yaw)
    sp, cp = math.sin(pitch), math.cos(pitch)
    fwd = (sy * cp, cy * cp, sp)
    right = (cy, -sy, 0.0)
    up = (-sy * sp, -cy * sp, cp)
    f_px = (w / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    scale = 262144.0 / f_px
    F = tuple(_rnd(524288.0 * c) for c in fwd)
    R = tuple(_rnd(scale * c) for c in right)
    U = tuple(_rnd(scale * c) for c in up)
    O = (_rnd(x * S), _rnd(y * S), _rnd(z * S))
    return (O, F, R, U, int(w), int(h))


def ray_camera(o, d):
    """A 1 x 1 camera whose single pixel ray is exactly (origin o, direction d)."""
    return (tuple(int(v) for v in o), tuple(int(v) for v in d), (0, 0, 0), (0, 0, 0), 1, 1)


def camera_array(cams):
    """Pack camera tuples into a CAMERA_DTYPE array."""
    a = np.zeros(len(cams), dtype=CAMERA_DTYPE)
    for i, (o, f, r, u, w, h) in enumerate(cams):
        a[i]["o"] = o
        a[i]["f"] = f
        a[i]["r"] = r
        a[i]["u"] = u
        a[i]["w"] = w
        a[i]["h"] = h
    return a


def _top(cells, x, y):
    h0, h1, h2, _ = unpack_cells(cells[int(y), int(x)])
    return int(h2) if int(h1) > int(h0) else int(h0)


# --- configurations --------------------------------------------------------

def config_c1():
    """256 x 256 grid (seed 1, 25 % slabs), one 320 x 240 camera, 60 deg FOV,
    at height 140 looking 35 deg down."""
    cells, _ = make_grid(256, 256, seed=1, slab_frac=0.25)
    cam = pose_to_camera(128.5, 16.5, 140.0, 0.0, -35.0, 60.0, 320, 240)
    return dict(name="C1", cells=cells, cams=camera_array([cam]))


def _c2_grid():
    return make_grid(2048, 2048, seed=2, slab_frac=0.40, n_walls=512)


def _c2_pose(cells, wall):
    H, W = cells.shape
    ys, xs = np.nonzero(~wall)
    d2 = (xs + 0.5 - 1024.5) ** 2 + (ys + 0.5 - 1024.5) ** 2
    k = int(np.argmin(d2))
    x, y = int(xs[k]), int(ys[k])
    h0 = int(cells[y, x] & 0xFF)
    yaw = 360.0 * float(unit_float(2, 6, 0))
    return x + 0.5, y + 0.5, h0 + 2.0, yaw


def config_c2(w=1920, h=1080):
    """2048 x 2048 grid with walls and 40 % cave slabs; one eye-level camera
    2 units above the floor, pitch 0, 90 deg FOV."""
    cells, wall = _c2_grid()
    x, y, z, yaw = _c2_pose(cells, wall)
    cam = pose_to_camera(x, y, z, yaw, 0.0, 90.0, w, h)
    return dict(name="C2", cells=cells, cams=camera_array([cam]), wall=wall)


def small_c2(w=240, h=135):
    """The C2 scene and pose at a reduced resolution."""
    return config_c2(w, h)


def c3_cameras(cells, seed=3, n=64, scale=1):
    """The 64 batched cameras: 16 x 3840x2160, 24 x 1920x1080, 24 x 640x360.

    Even-numbered cameras are top-down oblique (z in [150, 300], pitch in
    [-80, -30] deg), odd-numbered are eye level (2 units above the floor of
    their cell, pitch in [-5, 5] deg); yaw in [0, 360), hfov in [60, 90] deg.
    `scale` divides every resolution (for reduced-size parity runs).
    """
    H, W = cells.shape
    cams = []
    for i in range(n):
        if i < 16:
            w, h = 3840, 2160
        elif i < 40:
            w, h = 1920, 1080
        else:
            w, h = 640, 360
        w, h = max(1, w // scale), max(1, h // scale)
        u = [float(unit_float(seed, 7, 16 * i + k)) for k in range(6)]
        x = 64 + u[0] * (W - 128)
        y = 64 + u[1] * (H - 128)
        yaw = 360.0 * u[2]
        hfov = 60.0 + 30.0 * u[3]
        if i % 2 == 0:
            z = 150.0 + 150.0 * u[4]
            pitch = -80.0 + 50.0 * u[5]
        else:
            z = (cells[int(y), int(x)] & 0xFF) + 2.0
            pitch = -5.0 + 10.0 * u[5]
        cams.append(pose_to_camera(x, y, float(z), yaw, pitch, hfov, w, h))
    return camera_array(cams)


def config_c3(scale=1):
    """C2's grid with the 64 batched cameras (shadow rays on)."""
    cells, wall = _c2_grid()
    return dict(name="C3", cells=cells, cams=c3_cameras(cells, scale=scale), wall=wall)


def config_c4():
    """2048 x 16384 grid, seed 4, 30 % slabs (no walls)."""
    cells, _ = make_grid(2048, 16384, seed=4, slab_frac=0.30)
    return dict(name="C4", cells=cells)


def c4_waypoints(W, H, seed=4, n=16):
    xs = [256.0 + float(unit_float(seed, 8, 4 * k)) * (W - 512) for k in range(n)]
    ys = [1024.0 + k * (H - 2048) / (n - 1) + (float(unit_float(seed, 8, 4 * k + 1)) - 0.5) * 512
          for k in range(n)]
    alts = [float(uniform_int(seed, 8, 4 * k + 2, 3, 50)) for k in range(n)]
    return xs, ys, alts


def config_c4_frames(cells, n_frames=1000, w=1920, h=1080, hfov=90.0, seed=4):
    """Fly-through cameras: uniform Catmull-Rom through 16 seeded waypoints,
    altitude 3-50 above the local top, yaw along the tangent, pitch -10 deg."""
    H, W = cells.shape
    xs, ys, alts = c4_waypoints(W, H, seed)
    n = len(xs)

    def P(i):
        i = min(max(i, 0), n - 1)
        return xs[i], ys[i], alts[i]

    cams = []
    for f in range(n_frames):
        s = f * (n - 1) / max(1, n_frames - 1)
        k = min(int(s), n - 2)
        t = s - k
        p0, p1, p2, p3 = P(k - 1), P(k), P(k + 1), P(k + 2)
        pos, tan = [], []
        for a in range(2):
            c0, c1, c2, c3 = p0[a], p1[a], p2[a], p3[a]
            pos.append(0.5 * (2 * c1 + (-c0 + c2) * t + (2 * c0 - 5 * c1 + 4 * c2 - c3) * t * t
                              + (-c0 + 3 * c1 - 3 * c2 + c3) * t * t * t))
            tan.append(0.5 * ((-c0 + c2) + 2 * (2 * c0 - 5 * c1 + 4 * c2 - c3) * t
                              + 3 * (-c0 + 3 * c1 - 3 * c2 + c3) * t * t))
        x = min(max(pos[0], 0.5), W - 0.5)
        y = min(max(pos[1], 0.5), H - 0.5)
        alt = p1[2] + (p2[2] - p1[2]) * t
        z = _top(cells, x, y) + alt
        yaw = math.degrees(math.atan2(tan[0], tan[1]))
        cams.append(pose_to_camera(x, y, z, yaw, -10.0, hfov, w, h))
    return camera_array(cams)


PROTOCOL_PITCHES = (0.0, -30.0, -60.0, -90.0)
PROTOCOL_HEIGHT = {0.0: 6.0, -30.0: 60.0, -60.0: 120.0, -90.0: 200.0}


def protocol_cameras(cells, seed=12, w=1280, h=800, hfov=75.0, per_pitch=3):
    """The paper's protocol shape (its Section 4.3): three viewpoints at each
    pitch 0, -30, -60, -90 deg, 1280 x 800.  Positions and yaws are seeded
    over the grid (the paper's own viewpoints are locations in its level);
    each camera sits at a pitch-dependent height above its cell's top
    (6, 60, 120, 200 units); hfov 75 deg."""
    H, W = cells.shape
    cams = []
    for p_i, pitch in enumerate(PROTOCOL_PITCHES):
        for v in range(per_pitch):
            k = 3 * (per_pitch * p_i + v)
            x = 64.0 + float(unit_float(seed, 9, k)) * (W - 128)
            y = 64.0 + float(unit_float(seed, 9, k + 1)) * (H - 128)
            yaw = 360.0 * float(unit_float(seed, 9, k + 2))
            z = _top(cells, x, y) + PROTOCOL_HEIGHT[pitch]
            cams.append(pose_to_camera(x, y, z, yaw, pitch, hfov, w, h))
    return camera_array(cams)
