"""Footprints for the scattered renderer (inputs, not the method).

The scatter samples a camera-aligned ground footprint: longitudinal
coordinate s along fh (the horizontal direction 90 degrees left of the
camera's right vector R, i.e. its horizontal forward), lateral coordinate u
along R, |u| <= u_min + k_lat * |s|, s in [s_lo, s_hi].  This module chooses
those four numbers per camera: the rays of a 5 x 5 grid of image points
(corners and edges included) are followed to the plane z = 0 (or to the far
distance when they do not descend that far); s_lo, s_hi bound their (s, u);
k_lat is how fast the widest |u| grows from the image's bottom row of points
to its top row per unit of s (0 when it shrinks), and u_min the least value
that then holds every point; 5 % margins.  Terrain lies above z = 0, so what a
pixel can see lies within that bound.
"""

import numpy as np

S = 65536.0


def footprint_for(cam, far=600.0, margin=1.05):
    """(s_lo, s_hi, k_lat, u_min) as Python floats for one camera record."""
    O = np.asarray(cam["o"], np.float64) / S
    F = np.asarray(cam["f"], np.float64)
    R = np.asarray(cam["r"], np.float64)
    U = np.asarray(cam["u"], np.float64)
    w, h = int(cam["w"]), int(cam["h"])
    rl = np.hypot(R[0], R[1])
    if rl == 0.0:
        raise ValueError("the camera's right vector has no horizontal part")
    rh = np.array([R[0], R[1]]) / rl
    fh = np.array([-rh[1], rh[0]])
    ss, uu, rows = [], [], []
    for fa in np.linspace(-1.0, 1.0, 5):
        for fb in np.linspace(-1.0, 1.0, 5):
            d = F + fa * (w - 1) * R + fb * (h - 1) * U
            dl = np.linalg.norm(d)
            t_far = far / dl
            t = t_far
            if d[2] < 0:
                t = min(t_far, O[2] / -d[2])
            p = d[:2] * t
            ss.append(float(p @ fh))
            uu.append(float(p @ rh))
            rows.append(fb)
    ss, uu, rows = np.array(ss), np.abs(np.array(uu)), np.array(rows)
    s_lo = min(0.0, ss.min()) * margin - 1.0
    s_hi = max(1.0, ss.max() * margin + 1.0)
    top, bot = rows == 1.0, rows == -1.0
    ds = ss[top].mean() - ss[bot].mean()
    k_lat = max(0.0, (uu[top].max() - uu[bot].max()) / ds) if ds != 0.0 else 0.0
    u_min = float((uu - k_lat * np.abs(ss)).max())
    return float(s_lo), float(s_hi), float(k_lat * margin), float(max(u_min * margin, 0.0) + 1.0)


def footprints(cams, far=600.0):
    """float32 [n, 4] array of footprints, one row per camera."""
    return np.array([footprint_for(c, far) for c in cams], dtype=np.float32)
