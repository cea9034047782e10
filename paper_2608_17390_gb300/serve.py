"""Continuous-batching render server over one resident world.

The world (cells + pyramid) stays resident in one context.  Render requests
(a camera each) and edit requests (a rectangle of new cells) arrive over time.
The server loop:

  * admits arrived render requests in arrival order into a batch while output
    memory (a fixed byte budget) and a free lane (one CUDA stream per lane)
    allow, and launches the batch with one hf_render call on that lane: batches
    on different lanes run on the device at the same time, so requests that
    arrive while others are on the GPU start without waiting for them;
  * treats an edit as an ordering point: requests that arrived before it are
    admitted first; hf_edit then orders the cell copy and pyramid repair after
    every in-flight render and before every later one (the library's version
    rule, the paper's first-frame edit visibility of Section 4.4);
  * retires batches whose completion event has fired and frees their memory.

Latencies come from device timestamps: a reference event recorded at t0 on the
context stream maps every completion event to host time, so the measured frame
latency is (completion - arrival) without host polling delay, and the
edit-to-visible latency is (completion of the first render admitted after
the edit - the hf_edit call).
"""

import collections
import time

import numpy as np

from . import (HF_SHADOWS, alloc_outputs, hf_create, hf_destroy, hf_edit, hf_render, hf_sync,
               make_opts)

OUT_BYTES_PER_RAY = 14  # hit cell 4, layer 1, face 1, depth 4, rgba 4
SHADOW_BYTES_PER_RAY = 1


class Request:
    __slots__ = ("rid", "kind", "arrival", "cam", "edit", "rays", "admitted", "launched",
                 "done", "version", "outs", "lane", "batch_id", "call_time")

    def __init__(self, rid, kind, arrival, cam=None, edit=None):
        self.rid = rid
        self.kind = kind
        self.arrival = arrival
        self.cam = cam
        self.edit = edit
        self.rays = int(cam["w"]) * int(cam["h"]) if cam is not None else 0
        self.admitted = self.launched = self.done = self.call_time = None
        self.version = None
        self.outs = None
        self.lane = None
        self.batch_id = None


class Server:
    def __init__(self, cells, lanes=4, mem_bytes=4 << 30, max_batch=64, shadows=False,
                 opts=None):
        import torch

        self.torch = torch
        self.main = torch.cuda.Stream()
        self.ctx = hf_create(cells, stream=self.main.cuda_stream)
        self.lanes = [torch.cuda.Stream() for _ in range(lanes)]
        self.busy = [None] * lanes
        self.mem_budget = int(mem_bytes)
        self.mem_used = 0
        self.max_batch = max_batch
        self.shadows = shadows
        base = opts if opts is not None else make_opts()
        self.tile = (base.tile_w, base.tile_h, base.mip_start)
        self.flags = HF_SHADOWS if shadows else 0
        self.version = 0
        self.batches = 0
        self.max_inflight = 0

    def close(self):
        if self.ctx:
            hf_sync(self.ctx)
            hf_destroy(self.ctx)
            self.ctx = None

    def bytes_for(self, r):
        return r.rays * (OUT_BYTES_PER_RAY + (SHADOW_BYTES_PER_RAY if self.shadows else 0))

    def _launch(self, lane_i, batch):
        torch = self.torch
        lane = self.lanes[lane_i]
        with torch.cuda.stream(lane):
            for r in batch:
                r.outs = alloc_outputs(np.array([r.cam]), device="cuda", shadows=self.shadows)[0]
        cams = np.array([r.cam for r in batch])
        opts = make_opts(tile_w=self.tile[0], tile_h=self.tile[1], mip_start=self.tile[2],
                         flags=self.flags, stream=lane.cuda_stream)
        hf_render(self.ctx, cams, [r.outs for r in batch], opts)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(lane)
        self.busy[lane_i] = (ev, batch)
        self.max_inflight = max(self.max_inflight, sum(b is not None for b in self.busy))
        for r in batch:
            r.lane = lane_i
            r.batch_id = self.batches
        self.batches += 1

    def run(self, requests, keep_outputs=False, time_limit=None):
        """Serve `requests` (sorted by arrival, seconds from start).  Returns
        them with admitted / done times filled in (seconds from start)."""
        torch = self.torch
        ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ref.record(self.main)
        ref.synchronize()
        t0 = time.perf_counter()
        shift = clock_shift(torch, ref, self.lanes[0], lambda: time.perf_counter() - t0)
        edit_events = []
        pending = collections.deque(requests)
        queue = collections.deque()
        completed = []

        def retire(i, block=False):
            ev, batch = self.busy[i]
            if block:
                ev.synchronize()
            elif not ev.query():
                return False
            t_done = ref.elapsed_time(ev) / 1e3 + shift
            for r in batch:
                r.done = t_done
                self.mem_used -= self.bytes_for(r)
                if not keep_outputs:
                    r.outs = None
                completed.append(r)
            self.busy[i] = None
            return True

        while pending or queue or any(self.busy):
            now = time.perf_counter() - t0
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            for i in range(len(self.lanes)):
                if self.busy[i] is not None:
                    retire(i)
            while queue and queue[0].kind == "edit":
                r = queue.popleft()
                x0, y0, blk = r.edit
                r.call_time = time.perf_counter() - t0
                hf_edit(self.ctx, x0, y0, blk)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(self.main)  # after the edit's copy and repair
                edit_events.append((r, ev))
                self.version += 1
                r.version = self.version
                r.admitted = r.call_time
                r.done = r.call_time  # replaced by the device completion below
                completed.append(r)
            free = [i for i in range(len(self.lanes)) if self.busy[i] is None]
            if queue and free:
                batch = []
                while (queue and queue[0].kind == "render" and len(batch) < self.max_batch
                       and self.mem_used + self.bytes_for(queue[0]) <= self.mem_budget):
                    r = queue.popleft()
                    r.admitted = time.perf_counter() - t0
                    r.version = self.version
                    self.mem_used += self.bytes_for(r)
                    batch.append(r)
                if batch:
                    self._launch(free[0], batch)
                    continue
            if (queue and queue[0].kind == "render" and not any(self.busy)
                    and self.bytes_for(queue[0]) > self.mem_budget):
                raise ValueError("request %d needs more output memory than the whole budget"
                                 % queue[0].rid)
            if not queue and not pending:
                for i in range(len(self.lanes)):
                    if self.busy[i] is not None:
                        retire(i, block=True)
            elif not free or (queue and queue[0].kind == "render"):
                time.sleep(0)
        for i in range(len(self.lanes)):
            if self.busy[i] is not None:
                retire(i, block=True)
        for r, ev in edit_events:
            ev.synchronize()
            r.done = ref.elapsed_time(ev) / 1e3 + shift
        return completed


def clock_shift(torch, ref, stream, now, rounds=8):
    """Host time (seconds, on the clock `now`) of the CUDA event `ref`, which
    has already fired: each round trip records an event on the idle `stream`
    between two host readings, so before <= dev + shift <= after for its
    device time dev after `ref`.  Returns the middle of the intersected
    bracket (or of the narrowest round trip, if the brackets disagree)."""
    lo, hi, best = -1e30, 1e30, None
    ev = torch.cuda.Event(enable_timing=True)
    for _ in range(rounds):
        before = now()
        ev.record(stream)
        ev.synchronize()
        after = now()
        dev = ref.elapsed_time(ev) / 1e3
        lo, hi = max(lo, before - dev), min(hi, after - dev)
        if best is None or after - before < best[0]:
            best = (after - before, 0.5 * (before + after) - dev)
    return 0.5 * (lo + hi) if lo <= hi else best[1]


def run_native(ctx, records, lanes=8, max_batch=8, mem_bytes=4 << 30, shadows=False, opts=None):
    """The same request stream through the library's native serving loop
    (hf_serve_replay: the loop above, written in C++ behind the C ABI, with no
    Python between arrivals and launches).  Returns Request objects with the
    admitted / done / version fields filled in, for summarize()."""
    from . import hf_serve_replay

    base = opts if opts is not None else make_opts()
    res = hf_serve_replay(ctx, records, lanes=lanes, max_batch=max_batch, output_budget=mem_bytes,
                          flags=HF_SHADOWS if shadows else 0, tile_w=base.tile_w,
                          tile_h=base.tile_h, mip_start=base.mip_start)
    out = requests_from(records)
    for r, x in zip(out, res):
        r.admitted, r.done, r.version = float(x["admitted"]), float(x["done"]), int(x["version"])
        if r.kind == "edit":
            r.call_time = r.admitted
        else:
            r.batch_id = int(x["batch"])
    return out


def requests_from(records):
    """Request objects from the plain records of synth.poisson_requests."""
    out = []
    for i, rec in enumerate(records):
        if rec["kind"] == "edit":
            out.append(Request(i, "edit", rec["arrival"], edit=rec["edit"]))
        else:
            out.append(Request(i, "render", rec["arrival"], cam=rec["cam"]))
    return out


def summarize(completed, wall):
    """p50/p99 frame latency, p50/p99 edit-to-visible latency (ms), rays/s."""
    renders = [r for r in completed if r.kind == "render" and r.done is not None]
    edits = [r for r in completed if r.kind == "edit"]
    lat = np.array([(r.done - r.arrival) * 1e3 for r in renders])
    vis = []
    for e in edits:
        after = [r.done for r in renders if r.version is not None and r.version >= e.version]
        if after:
            first = min((r for r in renders if r.version is not None and r.version >= e.version),
                        key=lambda r: r.admitted)
            vis.append((first.done - e.call_time) * 1e3)
    vis = np.array(vis)
    rays = sum(r.rays for r in renders)
    span = max((r.done for r in renders), default=wall) - min((r.arrival for r in renders), default=0)
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    return {"renders": len(renders), "edits": len(edits),
            "frame_ms_p50": pct(lat, 50), "frame_ms_p99": pct(lat, 99),
            "edit_to_visible_ms_p50": pct(vis, 50), "edit_to_visible_ms_p99": pct(vis, 99),
            "rays_per_s": rays / span if span > 0 else None}
