"""The paper's image metrics (its Section 4.2), for scoring a renderer against
a reference rendering of the same cameras.

* see-through: the fraction of the reference's terrain pixels that the
  renderer leaves as background;
* covers-sky: the fraction of the reference's background pixels that the
  renderer fills;
* geometry: median and 95th percentile of |depth difference| over pixels
  where both have terrain;
* coherence: how many pixels (as a share of the image) have a depth at odds
  with the pixels around them in their 3 x 3 block, beyond the reference's
  own share of such pixels (never below zero).  The paper leaves "at odds"
  open; here a pixel is at odds when its
  terrain/background status differs from the majority of its 8 neighbours,
  or, for a terrain pixel among terrain neighbours, when its depth differs
  from the neighbourhood median by more than `rel_tol` of that median.
"""

import numpy as np


def incoherent_fraction(hit, depth, rel_tol=0.05):
    """Fraction of interior pixels that disagree with their 3 x 3 neighbourhood.

    hit: bool [h, w]; depth: float [h, w] (ignored where not hit)."""
    h, w = hit.shape
    if h < 3 or w < 3:
        return 0.0
    offs = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0)]
    core = (slice(1, h - 1), slice(1, w - 1))
    nb_hit = np.stack([hit[1 + dy:h - 1 + dy, 1 + dx:w - 1 + dx] for dy, dx in offs])
    d = np.where(hit, depth, np.nan)
    nb_d = np.stack([d[1 + dy:h - 1 + dy, 1 + dx:w - 1 + dx] for dy, dx in offs])
    majority_hit = nb_hit.sum(axis=0) >= 5
    status_bad = hit[core] != majority_hit
    with np.errstate(all="ignore"):
        med = np.nanmedian(nb_d, axis=0)
    depth_bad = hit[core] & majority_hit & (np.abs(depth[core] - med) > rel_tol * np.abs(med))
    return float((status_bad | depth_bad).mean())


def compare(ref_hit, ref_depth, hit, depth, rel_tol=0.05):
    """All four metrics for one image pair (2-D arrays of one camera)."""
    ref_hit = np.asarray(ref_hit, bool)
    hit = np.asarray(hit, bool)
    n_ref = int(ref_hit.sum())
    n_bg = int((~ref_hit).sum())
    both = ref_hit & hit
    err = np.abs(np.asarray(depth, np.float64)[both] - np.asarray(ref_depth, np.float64)[both])
    return {
        "see_through": float((ref_hit & ~hit).sum()) / n_ref if n_ref else 0.0,
        "covers_sky": float((~ref_hit & hit).sum()) / n_bg if n_bg else 0.0,
        "geometry_median": float(np.median(err)) if err.size else 0.0,
        "geometry_p95": float(np.percentile(err, 95)) if err.size else 0.0,
        "coherence": max(0.0, incoherent_fraction(hit, depth, rel_tol)
                         - incoherent_fraction(ref_hit, ref_depth, rel_tol)),
    }
