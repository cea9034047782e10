"""Shared helpers for the parity tests: run the CUDA path through the C ABI and
compare it with the oracle element by element.

Bars (from the method's accuracy target): hit cell, layer, face and shadow
bit-exact; depth within 1e-5 relative (0 only where the oracle has 0, +inf
where the oracle misses); colour within 1/255 per channel.
"""

import numpy as np

DEPTH_RTOL = 1e-5
RGBA_TOL = 1


def gpu_render(hf, ctx, cams, shadows=False, opts=None, fields=None):
    """Render through hf_render; returns a list of dicts of numpy arrays."""
    import torch

    kw = {} if fields is None else dict(fields=fields)
    outs = hf.alloc_outputs(cams, device="cuda", shadows=shadows, **kw)
    if opts is None:
        opts = hf.make_opts(flags=hf.HF_SHADOWS if shadows else 0)
    hf.hf_render(ctx, cams, outs, opts)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    res = []
    for o in outs:
        d = {}
        for k, t in o.items():
            a = t.cpu().numpy()
            if k in ("hit_cell", "rgba"):
                a = a.view(np.uint32)
            d[k] = a
        res.append(d)
    return res


def compare(gpu, orc, pix=None, shadows=False, what=""):
    """Assert GPU outputs (full image) match oracle outputs (full or at pix)."""
    sel = (lambda a: a) if pix is None else (lambda a: a[pix])
    for k in ("hit_cell", "layer", "face"):
        g, o = sel(gpu[k]), orc[k]
        bad = np.nonzero(g != o)[0]
        assert bad.size == 0, "%s %s mismatch at %d pixels, first %s: gpu %s oracle %s" % (
            what, k, bad.size, bad[:5], g[bad[:5]], o[bad[:5]])
    gd, od = sel(gpu["depth"]).astype(np.float64), orc["depth"]
    inf = np.isinf(od)
    assert (np.isinf(gd) == inf).all(), what + " depth miss pattern"
    fin = ~inf
    err = np.abs(gd[fin] - od[fin])
    tol = DEPTH_RTOL * np.abs(od[fin])
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, "%s depth: %d beyond 1e-5 rel, worst %g" % (
        what, bad.size, (err / np.maximum(np.abs(od[fin]), 1e-30)).max())
    g = sel(gpu["rgba"]).view(np.uint8).reshape(-1, 4).astype(np.int32)
    o = orc["rgba"].view(np.uint8).reshape(-1, 4).astype(np.int32)
    assert np.abs(g - o).max(initial=0) <= RGBA_TOL, what + " rgba beyond 1/255"
    if shadows:
        bad = np.nonzero(sel(gpu["shadow"]) != orc["shadow"])[0]
        assert bad.size == 0, "%s shadow mismatch at %d pixels" % (what, bad.size)


def sample_pixels(w, h, n, seed):
    """Seeded pixel sample: the four corners, the centre row and column ends,
    and n uniform pixels (sorted, unique)."""
    rng = np.random.default_rng(seed)
    pts = [0, w - 1, (h - 1) * w, h * w - 1, (h // 2) * w, (h // 2) * w + w - 1,
           w // 2, (h - 1) * w + w // 2]
    pts += rng.integers(0, w * h, n).tolist()
    return np.unique(np.array(pts, dtype=np.int64))
