"""The Section 4.2 image metrics on constructed image pairs."""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def metrics():
    import __graft_entry__

    __graft_entry__.build_library()
    from paper_2608_17390_gb300 import metrics as m

    return m


def _scene(h=40, w=60):
    yy, xx = np.mgrid[0:h, 0:w]
    hit = yy > h // 3
    depth = np.where(hit, 100.0 - yy, np.inf)
    return hit, depth


def test_identical_images_score_zero(metrics):
    hit, depth = _scene()
    m = metrics.compare(hit, depth, hit, depth)
    assert m == {"see_through": 0.0, "covers_sky": 0.0, "geometry_median": 0.0,
                 "geometry_p95": 0.0, "coherence": 0.0}


def test_coverage_decomposition(metrics):
    hit, depth = _scene()
    half = hit.copy()
    half[:, ::2] = False                     # drop half the terrain columns
    m = metrics.compare(hit, depth, half, np.where(half, depth, np.inf))
    assert m["see_through"] == pytest.approx(0.5, abs=0.02) and m["covers_sky"] == 0.0
    full = np.ones_like(hit)                 # fill every background pixel
    m = metrics.compare(hit, depth, full, np.where(hit, depth, 500.0))
    assert m["covers_sky"] == 1.0 and m["see_through"] == 0.0


def test_geometry_is_the_depth_error_where_both_hit(metrics):
    hit, depth = _scene()
    m = metrics.compare(hit, depth, hit, depth + 2.5)
    assert m["geometry_median"] == pytest.approx(2.5) and m["geometry_p95"] == pytest.approx(2.5)


def test_coherence_sees_speckle_not_smooth_offsets(metrics):
    hit, depth = _scene(80, 80)
    rng = np.random.default_rng(1)
    speck = hit.copy()
    holes = rng.random(hit.shape) < 0.05
    speck[holes & hit] = False               # isolated background pixels inside terrain
    m = metrics.compare(hit, depth, speck, np.where(speck, depth, np.inf))
    assert m["coherence"] > 0.03
    smooth = metrics.compare(hit, depth, hit, depth * 1.01)
    assert smooth["coherence"] == 0.0
