"""Seeded request streams for the serving loop: Poisson arrivals of render
requests of mixed sizes, interleaved with 64 x 64 crater edits."""

import numpy as np

from .cameras import camera_array, pose_to_camera
from .terrain import crater_edit

SERVING_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))


def poisson_requests(cells, n, rate, seed=5, edit_every=11, resolutions=SERVING_RESOLUTIONS):
    """n request records with exponential inter-arrival times at `rate` per
    second.  Every `edit_every`-th is a crater edit {kind, arrival, edit:
    (x0, y0, block)}, drawn against a host copy of the grid that is updated as
    edits are made (10 renders : 1 edit for edit_every = 11); the others are
    renders {kind, arrival, cam} at a resolution drawn uniformly from
    `resolutions`, from a random pose 3-50 units above the local top,
    yaw 0-360 deg, pitch -40..-5 deg, hfov 60-90 deg."""
    rng = np.random.default_rng(seed)
    H, W = cells.shape
    host = np.array(cells, dtype=np.uint32)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        if edit_every and i % edit_every == edit_every - 1:
            cx, cy = int(rng.integers(0, W)), int(rng.integers(0, H))
            x0, y0, blk = crater_edit(host, cx, cy)
            host[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk
            out.append({"kind": "edit", "arrival": t, "edit": (x0, y0, blk)})
            continue
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        x = float(rng.uniform(1.0, W - 1.0))
        y = float(rng.uniform(1.0, H - 1.0))
        c = int(host[int(y), int(x)])
        h0, h1, h2 = c & 0xFF, (c >> 8) & 0xFF, (c >> 16) & 0xFF
        top = h2 if h1 > h0 else h0
        z = top + float(rng.uniform(3.0, 50.0))
        cam = pose_to_camera(x, y, z, float(rng.uniform(0, 360)), float(rng.uniform(-40, -5)),
                             float(rng.uniform(60, 90)), w, h)
        out.append({"kind": "render", "arrival": t, "cam": camera_array([cam])[0]})
    return out
