"""Seeded input generators: ranges, validity, determinism, camera model."""

import math

import numpy as np

import synth


def _valid(cells):
    h0, h1, h2, mat = synth.unpack_cells(cells)
    slab = h1 > h0
    assert ((~slab) <= ((h1 == 0) & (h2 == 0))).all(), "no-slab cells must store h1 = h2 = 0"
    assert (h2[slab] >= h1[slab]).all()
    assert (mat <= 7).all()
    return h0, h1, h2, slab


def test_c1_grid_properties():
    c = synth.config_c1()
    cells = c["cells"]
    assert cells.shape == (256, 256) and cells.dtype == np.uint32
    h0, h1, h2, slab = _valid(cells)
    assert h0.min() >= 20 and h0.max() <= 120
    assert abs(slab.mean() - 0.25) < 0.005
    d1 = (h1 - h0)[slab]
    assert d1.min() >= 8 and d1.max() <= 40
    assert synth.grid_hash(cells) == synth.grid_hash(synth.config_c1()["cells"])


def test_walls_and_caves_grid():
    cells, wall = synth.make_grid(512, 384, seed=2, slab_frac=0.40, n_walls=40)
    h0, h1, h2, slab = _valid(cells)
    assert wall.any()
    assert set(np.unique(h0[wall]).tolist()) <= {0, 200}
    assert not slab[wall].any()
    assert (h0 == 200).sum() > 40 * 16 // 2


def test_noise_chunking_is_invisible():
    a = synth.value_noise(300, 70, seed=9, stream=0, base_period=32, chunk_rows=2048)
    b = synth.value_noise(300, 70, seed=9, stream=0, base_period=32, chunk_rows=7)
    assert (a == b).all()
    assert a.min() >= 0.0 and a.max() < 1.0


def test_crater_profile():
    cells, _ = synth.make_grid(128, 128, seed=5, slab_frac=0.5)
    x0, y0, blk = synth.crater_edit(cells, 60, 70)
    assert (x0, y0, blk.shape) == (28, 38, (64, 64))
    _valid(blk)
    old = synth.unpack_cells(cells[y0:y0 + 64, x0:x0 + 64])
    new = synth.unpack_cells(blk)
    yy, xx = np.mgrid[y0:y0 + 64, x0:x0 + 64]
    r2 = (xx - 60) ** 2 + (yy - 70) ** 2
    drop = old[0] - new[0]
    assert drop[r2 >= 1024].max() == 0
    assert new[0][32, 32] == max(0, old[0][32, 32] - 40)
    assert not (new[1] > new[0])[r2 < 400].any()
    keep = r2 >= 400
    assert (new[1][keep] == old[1][keep]).all() and (new[2][keep] == old[2][keep]).all()
    # clipped at the grid edge
    x0, y0, blk = synth.crater_edit(cells, 3, 125)
    assert (x0, y0, blk.shape) == (0, 93, (35, 35))


def _half_fov(cam):
    F = np.array(cam["f"], float)
    R = np.array(cam["r"], float)
    w = int(cam["w"])
    edge = F - w * R
    return math.degrees(math.acos(np.dot(F, edge) / (np.linalg.norm(F) * np.linalg.norm(edge))))


def test_fov_does_not_depend_on_resolution():
    """The focal length is fixed in pixels for a given width and FOV; the
    paper's evaluation section records a reference camera whose focal length
    was scaled by the image height, which changed the field of view with the
    resolution."""
    for hfov in (60.0, 90.0):
        for w, h in ((320, 240), (1920, 1080), (3840, 2160), (640, 1280)):
            cam = synth.camera_array([synth.pose_to_camera(10, 10, 50, 33.0, -20.0, hfov, w, h)])[0]
            assert abs(_half_fov(cam) - hfov / 2) < 0.5, (hfov, w, h)


def test_camera_axes():
    cam = synth.pose_to_camera(1.0, 2.0, 3.0, 0.0, 0.0, 90.0, 100, 50)
    o, F, R, U, w, h = cam
    assert o == (65536, 131072, 196608)
    assert F == (0, 524288, 0)            # yaw 0 looks along +y
    assert R[0] > 0 and R[1] == 0 and R[2] == 0   # right is +x
    assert U[2] > 0 and U[0] == 0 and U[1] == 0   # up is +z
    cam = synth.pose_to_camera(0, 0, 0, 90.0, -90.0, 90.0, 100, 50)
    assert cam[1][2] == -524288            # pitch -90 looks straight down


def test_c3_cameras_shape():
    c = synth.config_c3(scale=8)
    cams = c["cams"]
    assert len(cams) == 64
    assert (cams["w"][:16] == 480).all() and (cams["w"][40:] == 80).all()
    assert (cams["f"][0::2, 2] < 0).all()  # top-down half looks down
