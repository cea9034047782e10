"""Pins for the CPU oracle of the paper's fixed-step ray march (Section 3.1).

* On a flat plane every ray whose crossing lies at or before the last sample
  hits, and its depth lies in the bracket the four bisections leave:
  [t*, t* + dt/16] times |d| (dt = the sample spacing).
* A one-cell wall is skipped by most horizontal rays when the sample spacing
  (600 / 129 = 4.65 cells) exceeds its width -- the trade-off the paper
  acknowledges for its march: a feature narrower than the step can fall
  between two samples -- and found by every ray once the spacing is below
  one cell.
* Misses stay misses: no hit is made at the ground plane or outside the grid.
* A ray whose samples and bisection midpoints are exact in float32 pins the
  spacing t_end / (steps + 1), the clip at z = 0, the number of bisections
  and which end of the bracket they keep.
"""

import importlib.util
import math
import os

import numpy as np

import oracle
import synth

if os.environ.get("HF_MARCH_ORACLE"):
    # a planted-mistake copy of the march oracle (tests/test_oracle_mutations.py)
    _spec = importlib.util.spec_from_file_location("oracle._march_mutant",
                                                   os.environ["HF_MARCH_ORACLE"])
    march = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(march)
else:
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


def test_sample_spacing_and_bisection_closed_form():
    """One ray whose every sample and bisection midpoint is exact in float32.

    Origin height 129, direction (1, 0, -1) world units per unit t, floor of
    height 1 everywhere, far 600: the segment is clipped at z = 0, so
    t_end = 129 and the spacing t_end / (steps + 1) is exactly 1.  Samples
    t = 1 .. 128 lie at heights 128 .. 1; the first solid one is t = 128
    (z = 1, closed floor).  The four bisections of [127, 128] try 127.5,
    127.75, 127.875 and 127.9375, all above the floor, so the solid end stays
    at t = 128: depth = 128 * float32(sqrt 2), hit cell x = 10 + 128.  Any
    other spacing, clip or kept end moves the depth off this value."""
    W, H = 200, 4
    cells = _flat(W, H, 1)
    o = np.array([[10 * S + S // 2, 2 * S, 129 * S]], np.int64)
    d = np.array([[S, 0, -S]], np.int64)
    r = march.march(cells, o, d, steps=128, far=600.0, bisections=4)
    assert int(r["hit_cell"][0]) == 2 * W + 138
    assert int(r["layer"][0]) == 0
    assert float(r["depth"][0]) == float(np.float32(128.0) * np.sqrt(np.float32(2.0)))
    # three bisections leave [127.875, 128]: the solid end is still 128
    r3 = march.march(cells, o, d, steps=128, far=600.0, bisections=3)
    assert float(r3["depth"][0]) == float(r["depth"][0])
    # a floor of height 2: first solid sample t = 127 (z = 2); the midpoints
    # 126.5, 126.75, 126.875, 126.9375 lie above it
    r2 = march.march(_flat(W, H, 2), o, d, steps=128, far=600.0, bisections=4)
    assert float(r2["depth"][0]) == float(np.float32(127.0) * np.sqrt(np.float32(2.0)))


def test_bisection_converges_on_the_crossing():
    """Origin height 100.5 over a floor of height 1, same direction: t_end =
    100.5, spacing 100.5 / 129 (not exact), and the crossing z = 1 lies at
    t* = 99.5, between samples 127 and 128.  b bisections leave the solid end
    within spacing / 2^b after t*, and more bisections never move it away
    from t* or before it."""
    W, H = 200, 4
    cells = _flat(W, H, 1)
    o = np.array([[10 * S + S // 2, 2 * S, 100 * S + S // 2]], np.int64)
    d = np.array([[S, 0, -S]], np.int64)
    n = math.sqrt(2.0)
    dt = 100.5 / 129
    prev = None
    for b in (0, 1, 2, 4, 8):
        r = march.march(cells, o, d, bisections=b)
        depth = float(r["depth"][0])
        assert int(r["hit_cell"][0]) == 2 * W + 110  # x = 10.5 + t, t in [99.5, 100.28]
        assert 99.5 * n * (1 - 1e-6) <= depth <= (99.5 + dt / (1 << b)) * n * (1 + 1e-6), b
        if prev is not None:
            assert depth <= prev
        prev = depth


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
