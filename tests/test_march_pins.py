"""Pins for the CPU oracle of the paper's fixed-step ray march (Section 3.1).

* On a flat plane every ray whose crossing lies at or before the last sample
  hits, and its depth lies in the bracket the four bisections leave:
  [t*, t* + dt/16] times |d| (dt = the sample spacing).
* A one-cell wall is skipped by most horizontal rays when the sample spacing
  (600 / 129 = 4.65 cells) exceeds its width -- the method's trade-off the
  paper states ("a sample interval can still skip a thinner feature") -- and
  found by every ray once the spacing is below one cell.
* Misses stay misses: no hit is made at the ground plane or outside the grid.
"""

import math

import numpy as np

import oracle
import synth
from oracle import march

S = 65536


def _flat(W, H, h):
    return np.full((H, W), synth.pack_cells(h, 0, 0, 1), np.uint32)


def test_flat_plane_hits_inside_the_bisection_bracket():
    c = 30
    cells = _flat(400, 400, c)
    cam = synth.camera_array([synth.pose_to_camera(200.5, 200.5, 90.0, 20.0, -40.0, 80.0, 64, 48)])[0]
    res = march.march_camera(cells, cam, steps=128, far=600.0)
    dirs = oracle.ray_dirs(cam).astype(np.float64) / S
    o = np.array(cam["o"], np.float64) / S
    checked = 0
    for k in range(len(dirs)):
        d = dirs[k]
        n = math.sqrt((d * d).sum())
        t_end = 600.0 / n
        if d[2] < 0:
            t_end = min(t_end, -o[2] / d[2])
        dt = t_end / 129
        if d[2] >= 0:
            assert res["hit_cell"][k] == 0xFFFFFFFF
            continue
        t_star = (c - o[2]) / d[2]
        first = math.ceil(t_star / dt * (1 + 1e-6)) * dt  # first sample past the crossing
        px, py = o[0] + first * d[0], o[1] + first * d[1]
        inside = 0.5 < px < 399.5 and 0.5 < py < 399.5
        if t_star <= 128 * dt * (1 - 1e-5) and inside:
            assert res["hit_cell"][k] != 0xFFFFFFFF, k
            depth = float(res["depth"][k])
            assert t_star * n * (1 - 1e-5) <= depth <= (t_star + dt / 16) * n * (1 + 1e-5) + 1e-4
            checked += 1
    assert checked > 1000


def test_thin_wall_is_skipped_at_128_steps_and_found_with_fine_steps():
    W, H, wall = 700, 64, 330
    h0 = np.zeros((H, W), np.int64)
    h0[:, wall] = 250
    cells = synth.pack_cells(h0, 0, 0, 0)
    rng = np.random.default_rng(4)
    n = 300
    o = np.stack([rng.integers(10 * S, 100 * S, n), rng.integers(10 * S, 54 * S, n),
                  np.full(n, 10 * S)], 1)
    d = np.stack([np.full(n, S), rng.integers(-S // 50, S // 50, n), np.zeros(n, np.int64)], 1)
    exact = oracle.trace_rays(cells, o, d)
    assert (exact["hit_cell"] % W == wall).all()
    coarse = march.march(cells, o, d, steps=128)["hit_cell"]
    fine = march.march(cells, o, d, steps=4096)["hit_cell"]
    skipped = (coarse == 0xFFFFFFFF).mean()
    assert skipped > 0.5, skipped
    assert (fine % W == wall).all() and (fine != 0xFFFFFFFF).all()


def test_misses_stay_misses():
    # sea-level terrain under a camera: the segment is clipped at z = 0 and
    # its samples all lie above it, so nothing is hit (no ground-plane hit)
    cells = _flat(200, 200, 0)
    cam = synth.camera_array([synth.pose_to_camera(100.5, 100.5, 10.0, 0.0, -30.0, 60.0, 32, 24)])[0]
    res = march.march_camera(cells, cam)
    assert (res["hit_cell"] == 0xFFFFFFFF).all() and np.isinf(res["depth"]).all()
    # looking up from above every cell: nothing is solid up there
    cells = _flat(64, 64, 40)
    cam = synth.camera_array([synth.pose_to_camera(32.0, 32.0, 60.0, 0.0, 30.0, 60.0, 16, 12)])[0]
    res = march.march_camera(cells, cam)
    assert (res["hit_cell"] == 0xFFFFFFFF).all()


def test_march_hits_never_precede_the_exact_hit():
    """A solid sample is a solid point of the ray, so the march never stops
    before the exact first hit (up to float32 rounding of the sample point)."""
    cells, _ = synth.make_grid(256, 256, seed=1, slab_frac=0.25)
    cam = synth.camera_array([synth.pose_to_camera(128.5, 16.5, 140.0, 0.0, -35.0, 60.0, 80, 60)])[0]
    ex = oracle.render(cells, cam)
    mr = march.march_camera(cells, cam)
    both = (mr["hit_cell"] != 0xFFFFFFFF) & (ex["hit_cell"] != 0xFFFFFFFF)
    assert both.mean() > 0.5
    assert (mr["depth"][both] >= ex["depth"][both] * (1 - 1e-5) - 1e-3).all()
