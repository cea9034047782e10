"""Autotuner for the batched render: warp-tile shape and pyramid start level.

Tile shape and mip start change only how the exact traversal is scheduled,
never its result, so every candidate renders identical buffers; the tuner
keeps the fastest.  It times each candidate with CUDA events on the render
stream through the public API (hf_render), after one warm-up render, and
remembers the choice per (GPU name, grid size, resolution class).  The paper's
own tuning rule (its Section 5.6: the cheapest setting within one point of a
method's best error) has no error axis here -- every setting is exact -- so
the rule reduces to "fastest".
"""

import json
import os
import threading

import numpy as np

from . import HF_HOST_OUTPUTS, HF_MIP_AUTO, HF_SHADOWS, hf_info, hf_render, hf_sync, make_opts

DEFAULT_TILES = ((8, 4), (4, 8), (16, 2), (8, 8), (16, 4), (8, 16), (4, 16), (4, 32), (8, 32),
                 (4, 64))
# With HF_HOST_OUTPUTS the kernel's stores cross the host link, where a warp
# store of a short row piece costs nearly as much as a whole line: tiles whose
# rows are 32 pixels or wider keep those stores long.
HOST_TILES = ((16, 8), (32, 4), (64, 2), (64, 4), (128, 2), (256, 1))
DEFAULT_MIPS = (3, 4, 5, 6, 7, 8, 9)

_lock = threading.Lock()
_cache = {}


def resolution_class(cams):
    """Coarse size class of a batch: log2 of its mean pixel count."""
    px = [int(c["w"]) * int(c["h"]) for c in cams]
    return int(np.log2(max(1.0, float(np.mean(px)))))


def _key(ctx, cams, shadows, host_outputs=False):
    import torch

    info = hf_info(ctx)
    return (torch.cuda.get_device_name(info["device"]), info["width"], info["height"],
            resolution_class(cams), bool(shadows), bool(host_outputs))


def _time(ctx, cams, outs, opts, stream, reps):
    import torch

    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hf_render(ctx, cams, outs, opts)
        b.record(stream)
        hf_sync(ctx)
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def autotune(ctx, cams, outs, stream, shadows=False, tiles=None, mips=DEFAULT_MIPS,
             reps=3, cache_file=None, host_outputs=False):
    """Pick (tile_w, tile_h, mip_start) for this batch shape.

    ctx must order its work on `stream` (a torch.cuda.Stream); outs are the
    batch's output buffers (overwritten; pinned host tensors when
    host_outputs, which tunes and returns options with HF_HOST_OUTPUTS).
    tiles defaults to DEFAULT_TILES, or HOST_TILES for host outputs.  Returns
    (opts, table) where table lists (tile_w, tile_h, mip, ms) for every
    candidate timed (empty when the choice came from the cache)."""
    if tiles is None:
        tiles = HOST_TILES if host_outputs else DEFAULT_TILES
    key = _key(ctx, cams, shadows, host_outputs)
    with _lock:
        if not _cache and cache_file and os.path.exists(cache_file):
            try:
                for k, v in json.load(open(cache_file)).items():
                    _cache[tuple(json.loads(k))] = tuple(v)
            except (OSError, ValueError):
                pass
        hit = _cache.get(key)
    flags = (HF_SHADOWS if shadows else 0) | (HF_HOST_OUTPUTS if host_outputs else 0)
    if hit is not None:
        tw, th, mip = hit
        return make_opts(tile_w=tw, tile_h=th, mip_start=mip, flags=flags), []
    hf_render(ctx, cams, outs, make_opts(flags=flags, mip_start=HF_MIP_AUTO))
    hf_sync(ctx)
    # short renders are timed more often (a median over about 2 ms of
    # renders per candidate), so that launch jitter does not pick the tile
    t0 = _time(ctx, cams, outs, make_opts(flags=flags, mip_start=HF_MIP_AUTO), stream, 1)
    if t0 < 1.0:
        reps = int(min(25, max(reps, np.ceil(2.0 / max(t0, 0.01)))))
    table = []
    for tw, th in tiles:
        for mip in mips:
            ms = _time(ctx, cams, outs, make_opts(tile_w=tw, tile_h=th, mip_start=mip, flags=flags),
                       stream, reps)
            table.append((tw, th, mip, ms))
    tw, th, mip, _ = min(table, key=lambda r: r[3])
    with _lock:
        _cache[key] = (tw, th, mip)
        if cache_file:
            tmp = cache_file + ".tmp"
            with open(tmp, "w") as f:
                json.dump({json.dumps(list(k)): list(v) for k, v in _cache.items()}, f)
            os.replace(tmp, cache_file)
    return make_opts(tile_w=tw, tile_h=th, mip_start=mip, flags=flags), table
