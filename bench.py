"""Benchmark: primary rays/s of the batched exact ray cast on one GB300.

One step = one whole pass of the hot path over one batch: a 64 x 64 crater
edit with incremental pyramid repair, then one batched render of the 64
cameras of the batched-cameras workload (16 x 3840x2160, 24 x 1920x1080,
24 x 640x360, half top-down, half eye level) with one shadow ray per hit, on
the 2048 x 2048 walls-and-caves grid.  value = primary rays / s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hf|reference]
                  [--workload c3|c2|c4|c1|c5]

--workload c5 runs the serving loop instead and prints its latency line.

Under torchrun each rank renders its own copy of the batch (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def _peak_sm_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------- ncu traffic

TRACE_SOURCES = ("paper_2608_17390_gb300/csrc/hf_trace.cu", "paper_2608_17390_gb300/csrc/hf_internal.h")


def trace_source_hash():
    """Hash of the trace kernel's code: its sources with comments and blank
    lines removed, so that the committed ncu figures stay attached to the
    code they were measured on across edits of comments only."""
    import hashlib
    import re

    h = hashlib.sha256()
    for rel in TRACE_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(l.rstrip() for l in src.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def _profile_fields(workload):
    path = os.path.join(ROOT, "profiles", "trace_batched_%s.md" % workload)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_source_sha256") != trace_source_hash():
        return None
    return fields


def _profiled(workload, key, tile, mip):
    """One per-launch figure from the committed ncu summary of this workload,
    for the launch configuration (tile, mip start) given: the summary's main
    capture when its configuration is this one, else a `key@tile/mip` line
    taken for another configuration.  None when there is none, or when the
    kernel source changed since the counters were taken."""
    f = _profile_fields(workload)
    if not f:
        return None
    if f.get("launch_tile") == tile and f.get("launch_mip_start") == str(mip) and key in f:
        v = f[key]
    else:
        v = f.get("%s@%s/%s" % (key, tile, mip))
    try:
        return float(v) if v is not None else None
    except ValueError:
        return None


def _alu_roofline(workload, rays, render_ms, tile, mip, sm_count, sm_mhz):
    """Instruction-issue roofline of the trace kernel: warp instructions per
    primary ray (ncu, full-size launch of the same source and launch
    configuration) times this launch's rays, over the live render time,
    against SMs x 4 schedulers x 1 instruction/cycle x the SM clock."""
    per_ray = _profiled(workload, "warp_instructions_per_primary_ray", tile, mip)
    if per_ray is None:
        return None
    achieved = per_ray * rays / (render_ms / 1e3) / 1e12
    peak = sm_count * 4 * sm_mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T warp-instr/s",
            "frac": achieved / peak, "warp_instructions_per_primary_ray": per_ray,
            "peak_source": "%d SMs x 4 schedulers x 1 instr/cycle x %.0f MHz" % (sm_count, sm_mhz)}


def _profiled_traffic(workload, rays, tile, mip):
    """DRAM bytes (read + write) per launch of the trace kernel, from the
    committed ncu summary of this workload: its measured bytes per ray for
    this launch configuration times the rays of one launch here.  None when
    there is no such figure, or when the kernel source changed since the
    counters were taken."""
    per_ray = _profiled(workload, "dram_bytes_per_ray", tile, mip)
    return None if per_ray is None else per_ray * rays


# ------------------------------------------------------------------ workloads

def workload(name, rank=0, scale=1, frames_per_step=100):
    import synth

    if name == "c3":
        cfg = synth.config_c3(scale=scale)
        return dict(name="C3 batched cameras: 2048x2048 walls+caves grid (seed 2), 64 cameras "
                         "(16x3840x2160, 24x1920x1080, 24x640x360), shadow rays on, one 64x64 "
                         "crater edit + incremental pyramid repair per step",
                    cells=cfg["cells"], cams=cfg["cams"], shadows=True, edit=True)
    if name == "c2":
        cfg = synth.config_c2()
        return dict(name="C2 eye-level horizon: 2048x2048 walls+caves grid, one 1920x1080 camera "
                         "2 units above the floor, pitch 0, hfov 90",
                    cells=cfg["cells"], cams=cfg["cams"], shadows=False, edit=False)
    if name == "c1":
        cfg = synth.config_c1()
        return dict(name="C1 small: 256x256 grid, one 320x240 camera", cells=cfg["cells"],
                    cams=cfg["cams"], shadows=False, edit=False)
    if name == "c4":
        cells = synth.config_c4()["cells"]
        return dict(name="C4 large world: 2048x16384 grid (seed 4, 30%% slabs), 1000-frame "
                         "1920x1080 fly-through; one step = %d frames in one batch" % frames_per_step,
                    cells=cells, cams=synth.config_c4_frames(cells, 1000), shadows=False,
                    edit=False, frames_per_step=frames_per_step)
    if name == "c4pair":
        cells = synth.pairify(synth.config_c4()["cells"] & np.uint32(0x07FFFFFF))
        return dict(name="C4 large world in paired 2-byte texels (64 MiB of cells): 2048x16384 "
                         "grid (seed 4, 30%% slabs, slab pairs sharing one column), 1000-frame "
                         "1920x1080 fly-through; one step = %d frames in one batch" % frames_per_step,
                    cells=cells, texels=synth.encode_pairs(cells),
                    cams=synth.config_c4_frames(cells, 1000), shadows=False, edit=False,
                    frames_per_step=frames_per_step)
    raise SystemExit("unknown workload " + name)


def n_rays(cams):
    return int(sum(int(c["w"]) * int(c["h"]) for c in cams))


# -------------------------------------------------------------- clocks probe

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------- CPU oracle

def cpu_model():
    """The host CPU's model name (lscpu), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def _pixel_sample(cams, frac, seed):
    """Seeded pixel indices per camera: about frac of each camera's pixels (at
    least 16), so the sample mixes views, resolutions and ray lengths as the
    whole workload does."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        n = int(c["w"]) * int(c["h"])
        k = max(16, min(n, int(round(frac * n))))
        out.append(np.unique(rng.integers(0, n, k)).astype(np.uint32))
    return out


def cpu_oracle_sample(wl, budget_s=15.0, seed=0, threads=None):
    """Oracle rays/s on a bounded, seeded sample of the workload: the same
    fraction of every camera's pixels, one oracle call per camera on
    `threads` host threads (all cores by default).  A short calibration pass
    picks the fraction so that the measured pass takes about budget_s."""
    import oracle

    cores = threads or os.cpu_count() or 1
    cams = wl["cams"]
    total = n_rays(cams)

    def run(frac, sd):
        pix = _pixel_sample(cams, frac, sd)
        t0 = time.perf_counter()
        for c, p in zip(cams, pix):
            oracle.render(wl["cells"], c, shadows=wl["shadows"], pix=p, nthreads=cores)
        return sum(len(p) for p in pix), time.perf_counter() - t0

    n0, t0 = run(min(1.0, 1.0e5 * cores / total), seed + 7919)
    frac = min(1.0, budget_s * (n0 / t0) / total)
    done, dt, passes = 0, 0.0, 0
    while passes == 0 or (frac == 1.0 and dt < 0.5 * budget_s and passes < 10000):
        # a workload smaller than the budget is sampled whole, pass after pass
        d, t = run(frac, seed + passes)
        done, dt, passes = done + d, dt + t, passes + 1
    return {"value": done / dt, "unit": "primary rays/s", "cores": cores, "kind": "oracle",
            "sample": "%d seeded pixels (%.3g%% of each of the %d cameras' pixels, one oracle "
                      "call per camera%s)%s, %.1f s" % (
                          done, 100 * frac, len(cams),
                          ", %d passes" % passes if passes > 1 else "",
                          " with shadow rays" if wl["shadows"] else "", dt)}


def cpu_baseline(wl, budget_s=15.0):
    """The host-core oracle figure for the bench line: all cores, plus the
    same sample design on one core (a third of the budget), with the CPU
    model and core count."""
    allc = cpu_oracle_sample(wl, budget_s=budget_s)
    one = cpu_oracle_sample(wl, budget_s=budget_s / 3.0, seed=1, threads=1)
    allc["single_core"] = {"value": one["value"], "unit": one["unit"], "sample": one["sample"]}
    allc["nproc"] = os.cpu_count()
    allc["cpu_model"] = cpu_model()
    return allc


# ---------------------------------------------------------------- GPU arm

def run_hf(args):
    import torch

    import __graft_entry__

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        if local == 0:  # one build per node; the other ranks wait for it
            __graft_entry__.build_library()
        dist.barrier()
    else:
        torch.cuda.set_device(0)
        __graft_entry__.build_library()
    import paper_2608_17390_gb300 as hf
    import synth

    wl = workload(args.workload, rank, args.scale, args.frames_per_step)
    if args.scale != 1:
        wl["name"] += " (resolutions divided by %d)" % args.scale
    cells = wl["cells"].copy()
    cams_all = wl["cams"]
    fps = wl.get("frames_per_step")
    stream = torch.cuda.Stream()
    if "texels" in wl:
        ctx = hf.hf_create_pairs(wl["texels"], stream=stream.cuda_stream)
    else:
        ctx = hf.hf_create(cells, stream=stream.cuda_stream)
    info = hf.hf_info(ctx)
    flags = hf.HF_SHADOWS if wl["shadows"] else 0

    def step_cams(i):
        if fps:
            k = (i * fps) % len(cams_all)
            return cams_all[k:k + fps]
        return cams_all

    max_cams = step_cams(0)
    outs = hf.alloc_outputs(max_cams, device="cuda", shadows=wl["shadows"])
    tuned = None
    if args.mip == 0xFFFFFFFF and not args.tile_w and not args.tile_h and not args.no_tune:
        from paper_2608_17390_gb300.autotune import autotune

        opts, table = autotune(ctx, max_cams, outs, stream, shadows=wl["shadows"], reps=2)
        tuned = {"candidates": len(table), "best_ms": min(r[3] for r in table) if table else None}
    else:
        opts = hf.make_opts(flags=flags, mip_start=args.mip, tile_w=args.tile_w,
                            tile_h=args.tile_h)
    tile_w, tile_h, mip_start = opts.tile_w or 8, opts.tile_h or 4, opts.mip_start
    rng = np.random.default_rng(1234)
    H, W = cells.shape

    def draw_edit():
        cx, cy = int(rng.integers(0, W)), int(rng.integers(0, H))
        x0, y0, blk = synth.crater_edit(cells, cx, cy)
        if "texels" in wl:  # a paired-texel world is edited in whole, representable pairs
            h, w = blk.shape
            xa, xb = x0 & ~1, (x0 + w + 1) & ~1
            full = cells[y0:y0 + h, xa:xb].copy()
            full[:, x0 - xa:x0 - xa + w] = blk
            x0, blk = xa, synth.pairify(full)
        return x0, y0, blk

    def do_edit(pre=None):
        """One crater: drawn here (or given, drawn before a timed region), then
        uploaded and repaired by hf_edit."""
        if ws > 1:
            # the replicas' one exchange step: rank 0 draws the crater, every
            # rank receives it and applies it to its own world
            from paper_2608_17390_gb300.replicas import replicated_edit

            replicated_edit(draw_edit() if rank == 0 else None, cells, src=0, device="cuda",
                            apply=lambda x0, y0, b: hf.hf_edit(ctx, x0, y0, b))
            return
        x0, y0, blk = pre if pre is not None else draw_edit()
        hf.hf_edit(ctx, x0, y0, blk)
        cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]] = blk

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def _ev_ms(fn, reps=5):
        ts = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            hf.hf_sync(ctx)
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    # rows a2 / a3: full pyramid build, and one crater edit (H2D of the rect +
    # incremental repair), each on the context stream, L2 flushed before
    build_ms = _ev_ms(lambda: hf.hf_rebuild(ctx))
    edit_ms = _ev_ms(do_edit)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def one_step(i, rec=None):
        cams = step_cams(i)
        if rec:
            rec[0].record(stream)
        if wl["edit"]:
            do_edit()
        if rec:
            rec[1].record(stream)
        hf.hf_render(ctx, cams, outs[:len(cams)], opts)
        if rec:
            rec[2].record(stream)

    # untimed: fetch counters for the algorithmic bytes of one render
    sopts = hf.make_opts(flags=flags | hf.HF_STATS, mip_start=mip_start, tile_w=tile_w,
                         tile_h=tile_h)
    hf.hf_stats(ctx)
    hf.hf_render(ctx, max_cams, outs[:len(max_cams)], sopts)
    st = hf.hf_stats(ctx)
    # with shadow rays that render built the per-cell shadow bounds: a full
    # rebuild now also rebuilds them
    rebuild_ms = _ev_ms(lambda: hf.hf_rebuild(ctx)) if wl["shadows"] else None
    for i in range(args.warmup):
        one_step(i)
    hf.hf_sync(ctx)
    torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device())
    if rank == 0:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    render_ms, step_ms = [], []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)  # evict L2 between timed steps (256 MiB > L2)
        one_step(args.warmup + i, ev[i])
    hf.hf_sync(ctx)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ck = clocks.stop() if rank == 0 else None
    for a, b, c in ev:
        step_ms.append(a.elapsed_time(c))
        render_ms.append(b.elapsed_time(c))
    total_ms = float(np.sum(step_ms))
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    rays_step = sum(n_rays(step_cams(args.warmup + i)) for i in range(args.steps)) / args.steps
    value = rays_step * args.steps * ws / (total_ms / 1e3)

    # plain: one launch per camera, same accuracy, same stream, L2 flushed;
    # its tile shape is chosen for it (one render per candidate), since the
    # batched kernel's choice need not suit one launch per camera
    plain = plain_tile = None
    if not args.no_plain:
        def plain_ms(tw, th, reps):
            popts = hf.make_opts(flags=flags | hf.HF_PLAIN, mip_start=mip_start, tile_w=tw,
                                 tile_h=th)
            pms = []
            for i in range(reps):
                with torch.cuda.stream(stream):
                    flush.fill_(7)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                hf.hf_render(ctx, max_cams, outs[:len(max_cams)], popts)
                b.record(stream)
                hf.hf_sync(ctx)
                pms.append(a.elapsed_time(b))
            return float(np.median(pms))

        cands = [(tile_w, tile_h)] + [t for t in ((8, 4), (4, 8), (8, 8), (4, 16), (8, 16), (4, 32),
                                                   (8, 32), (4, 64)) if t != (tile_w, tile_h)]
        plain_ms(*cands[0], 1)  # warm-up
        plain_tile = min(cands, key=lambda t: plain_ms(t[0], t[1], 1))
        plain = n_rays(max_cams) / (plain_ms(*plain_tile, max(1, min(3, args.steps))) / 1e3)

    # end to end through the public API with host buffers: host camera records
    # and edit cells in, every output field back in pinned host memory, timed
    # on the host clock around the whole call.  Two library paths, the faster
    # reported: the kernel writes the pinned host buffers itself
    # (HF_HOST_OUTPUTS), or renders chunks into device staging that the copy
    # engine moves back while later chunks render (HF_HOST_STAGED).  For
    # context: device buffers, then one copy per output field (each field of
    # all cameras is one allocation, see alloc_outputs).
    e2e = e2e_copy = None
    if not args.no_e2e:
        host = hf.alloc_outputs(max_cams, device="pinned", shadows=wl["shadows"])
        cam_bytes = max_cams.nbytes
        out_bytes = sum(v.numel() * v.element_size() for o in host for v in o.values())
        if tuned is not None:
            from paper_2608_17390_gb300.autotune import autotune

            hopts, htable = autotune(ctx, max_cams, host, stream, shadows=wl["shadows"], reps=2,
                                     mips=(mip_start,), host_outputs=True)
        else:
            hopts = hf.hf_render_opts.from_buffer_copy(opts)
            hopts.flags |= hf.HF_HOST_OUTPUTS

        sopts = hf.hf_render_opts.from_buffer_copy(opts)
        sopts.flags |= hf.HF_HOST_STAGED

        def e2e_time(via_host):
            ems = []
            for i in range(max(1, min(5, args.steps))):
                with torch.cuda.stream(stream):
                    flush.fill_(9)
                # the crater is an input: drawn on the host before the timed region
                # (on one GPU; under torchrun its broadcast is part of the step)
                pre = draw_edit() if wl["edit"] and ws == 1 else None
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if wl["edit"]:
                    do_edit(pre)
                if via_host == "staged":
                    hf.hf_render(ctx, max_cams, host, sopts)
                elif via_host:
                    hf.hf_render(ctx, max_cams, host, hopts)
                else:
                    hf.hf_render(ctx, max_cams, outs[:len(max_cams)], opts)
                    with torch.cuda.stream(stream):
                        for k in outs[0]:
                            host[0][k].untyped_storage().copy_(outs[0][k].untyped_storage(),
                                                               non_blocking=True)
                stream.synchronize()
                ems.append(time.perf_counter() - t0)
            return n_rays(max_cams) / float(np.median(ems))

        e2e_copy = e2e_time(False)
        e2e_time("staged")  # first call allocates the staging
        direct, staged = e2e_time(True), e2e_time("staged")
        paths = {"direct": ("hf_render with HF_HOST_OUTPUTS: the kernel writes pinned host buffers "
                            "(tile %dx%d)" % (hopts.tile_w or 8, hopts.tile_h or 4), direct),
                 "staged": ("hf_render with HF_HOST_STAGED: chunks rendered to device staging, each "
                            "copied back while the next renders", staged)}
        best = max(paths, key=lambda k: paths[k][1])
        e2e = {"value": paths[best][1], "unit": "primary rays/s",
               "h2d_bytes_per_step": int(cam_bytes + (64 * 64 * 4 if wl["edit"] else 0)),
               "d2h_bytes_per_step": int(out_bytes), "path": paths[best][0],
               "host_outputs_direct": direct, "host_staged": staged, "render_then_copy": e2e_copy}

    hf.hf_destroy(ctx)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    hbm, src = _peaks()
    rays = st["rays"]
    out_b = rays * (14 + (1 if wl["shadows"] else 0))
    fetch_b = 4 * (st["node_fetches"] + st["cell_fetches"] + st["shadow_fetches"])
    alg_bytes = fetch_b + out_b
    r_ms = float(np.mean(render_ms))
    achieved = alg_bytes / (r_ms / 1e3) / 1e9
    traffic = _profiled_traffic(args.workload, rays, "%dx%d" % (tile_w, tile_h), mip_start)
    line = {
        "metric": "primary rays/s (batched, exact two-interval height-field ray cast)",
        "value": value, "unit": "primary rays/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
        "data": "synthetic (seeded value-noise terrain standing in for the paper's Fostral level)",
        "config": {"workload": wl["name"], "rays_per_step": int(rays_step),
                   "grid": "%dx%d" % (W, H), "l2": "flushed between steps (256 MiB write)",
                   "mip_start": "library default" if mip_start == 0xFFFFFFFF else mip_start,
                   "tile": "%dx%d" % (tile_w, tile_h),
                   "autotuned": tuned,
                   "world_bytes": info["cell_bytes"] + info["pyramid_bytes"]},
        "plain_rays_per_s": plain,
        "plain_tile": ("%dx%d" % plain_tile) if plain_tile else None,
        "batched_over_plain": (value / ws / plain) if plain else None,
        "render_ms": r_ms,
        "pyramid_build_ms": build_ms,
        "pyramid_and_sun_bounds_build_ms": rebuild_ms,
        "edit_repair_ms": edit_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": src,
                     "bytes_per_ray": alg_bytes / max(rays, 1),
                     "note": "algorithmic bytes = 4 B x (pyramid nodes + cells + shadow-ray "
                             "fetches, counted in-kernel) + %d B output per ray; most fetches "
                             "are L2/L1 hits" % (14 + (1 if wl["shadows"] else 0))},
        "alu_roofline": _alu_roofline(args.workload, rays, r_ms, "%dx%d" % (tile_w, tile_h),
                                      mip_start, info["sm_count"],
                                      (ck or {}).get("sm_mhz") or _peak_sm_mhz()),
        "fetches_per_ray": (st["node_fetches"] + st["cell_fetches"]) / max(rays, 1),
        # per step: the render, and for a crater the pyramid repair plus, once
        # the shadow bounds exist (shadow rays toward the default sun), their repair
        "gpu_launches": args.steps * (1 + ((2 if wl["shadows"] else 1) if wl["edit"] else 0)),
        "clocks": ck,
        "e2e": e2e,
    }
    if not args.no_cpu and ws == 1:  # the host-core oracle sample: rank 0 at N = 1 only
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_seconds)
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# serving lanes (streams) and requests per batch: swept at 70 % and 100 % load
# (lanes 2/4/8/16, batches up to 8/32); 8 lanes of up to 8 requests gave the
# lowest p99 frame latency at both loads
SERVE_LANES, SERVE_MAX_BATCH = 8, 8


def run_serve(args):
    """Serving loop on the large world: p50/p99 frame and edit-to-visible
    latency at ~70 % and ~100 % of the measured batched capacity."""
    import torch

    import __graft_entry__

    ws, rank, local = _dist()
    torch.cuda.set_device(local if ws > 1 else 0)
    __graft_entry__.build_library()
    import paper_2608_17390_gb300 as hf
    from paper_2608_17390_gb300 import serve
    import synth

    cells = synth.config_c4()["cells"]
    srv = serve.Server(cells, lanes=SERVE_LANES, mem_bytes=4 << 30, max_batch=SERVE_MAX_BATCH)
    # capacity: one batched render of 64 representative requests
    probe = [r for r in synth.poisson_requests(cells, 72, 1.0, seed=99) if r["kind"] == "render"]
    cams = np.array([r["cam"] for r in probe])
    outs = hf.alloc_outputs(cams)
    ms = []
    for _ in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(srv.main)
        hf.hf_render(srv.ctx, cams, outs, hf.make_opts(stream=srv.main.cuda_stream))
        b.record(srv.main)
        hf.hf_sync(srv.ctx)
        ms.append(a.elapsed_time(b))
    cap_rays = n_rays(cams) / (float(np.median(ms[1:])) / 1e3)
    mean_rays = n_rays(cams) / len(cams)
    cap_req = cap_rays / mean_rays * 10.0 / 11.0  # requests/s incl. 1 edit per 10 renders
    del outs
    # each load: the library's native loop (hf_serve_replay, reported), then the
    # Python loop over the same request stream (for comparison)
    results, py_results = {}, {}
    all_clocks = Clocks(torch.cuda.current_device())
    all_clocks.start()
    for load in (0.7, 1.0):
        records = synth.poisson_requests(cells, args.serve_requests, load * cap_req,
                                         seed=int(load * 100))
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        t0 = time.perf_counter()
        done = serve.run_native(srv.ctx, records, lanes=SERVE_LANES, max_batch=SERVE_MAX_BATCH,
                                mem_bytes=4 << 30)
        st = serve.summarize(done, time.perf_counter() - t0)
        st["clocks"] = clocks.stop()
        st["offered_requests_per_s"] = load * cap_req
        st["batches"] = len({r.batch_id for r in done if r.kind == "render"})
        results["load_%d%%" % int(load * 100)] = st
        b0 = srv.batches
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        t0 = time.perf_counter()
        done = srv.run(serve.requests_from(records))
        st = serve.summarize(done, time.perf_counter() - t0)
        st["clocks"] = clocks.stop()
        st["batches"] = srv.batches - b0
        st["max_inflight_batches"] = srv.max_inflight
        py_results["load_%d%%" % int(load * 100)] = st
    ck = all_clocks.stop()
    srv.close()
    if rank != 0:
        return
    hi = results["load_100%"]
    line = {"metric": "p50/p99 frame and edit-to-visible latency, serving loop (continuous "
                      "batching, 10 renders : 1 edit)",
            "serving_loop": "native (hf_serve_replay); loads_python_loop: the same streams "
                            "through the Python loop (serve.Server)",
            "value": hi["frame_ms_p99"], "unit": "ms (p99 frame latency at ~100% load)",
            "n_gpus": ws, "steps": args.serve_requests, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": "C5 serving: 2048x16384 grid resident, Poisson render "
                                   "requests (640x360..3840x2160, random poses) with a 64x64 "
                                   "crater edit every 11th request", "lanes": SERVE_LANES,
                       "output_memory_budget_bytes": 4 << 30, "max_batch": SERVE_MAX_BATCH},
            "capacity_rays_per_s": cap_rays, "capacity_requests_per_s": cap_req,
            "loads": results, "loads_python_loop": py_results, "clocks": ck}
    print(json.dumps(line))


def run_protocol(args):
    """The paper's protocol shape (its Sections 4.3 and 5.2): 12 viewpoints at
    pitch 0 / -30 / -60 / -90, 1280x800, far 600, on the large world.  Times
    the exact cast and the paper's fixed-step march (steady-state frames and
    one batched launch of all 12 views) and scores the march against the exact
    cast with the Section 4.2 metrics."""
    import torch

    import __graft_entry__

    torch.cuda.set_device(0)
    __graft_entry__.build_library()
    import paper_2608_17390_gb300 as hf
    from paper_2608_17390_gb300 import metrics
    import synth

    cells = synth.config_c4()["cells"]
    cams = synth.protocol_cameras(cells)
    stream = torch.cuda.Stream()
    ctx = hf.hf_create(cells, stream=stream.cuda_stream)
    fields = ("hit_cell", "layer", "depth")
    outs = hf.alloc_outputs(cams, fields=fields)

    def ev_ms(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for r in range(reps):
            fn(r)
        b.record(stream)
        hf.hf_sync(ctx)
        return a.elapsed_time(b) / reps

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    exact = hf.make_opts(stream=stream.cuda_stream)
    frame = lambda r: hf.hf_render(ctx, cams[r % 12:r % 12 + 1], outs[r % 12:r % 12 + 1], exact)
    batch = lambda r: hf.hf_render(ctx, cams, outs, exact)
    ev_ms(frame, 24)
    res = {"exact": {"frame_ms": ev_ms(frame, 40), "batch12_ms": ev_ms(batch, 10)}}
    ref = [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]

    def by_pitch():
        """Section 4.2 metrics of the current outputs against the exact cast
        (clipped at the same far distance), averaged over the views of a pitch."""
        got = [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]
        per_pitch = {}
        for p_i, pitch in enumerate(synth.PROTOCOL_PITCHES):
            ms = []
            for v in range(3):
                i = 3 * p_i + v
                h, w = int(cams[i]["h"]), int(cams[i]["w"])
                rd = ref[i]["depth"].reshape(h, w).astype(np.float64)
                rh = np.isfinite(rd) & (rd <= 600.0)
                gd = got[i]["depth"].reshape(h, w).astype(np.float64)
                ms.append(metrics.compare(rh, rd, np.isfinite(gd), gd))
            per_pitch["%d" % int(pitch)] = {k: float(np.mean([m[k] for m in ms])) for k in ms[0]}
        return per_pitch

    for st in (16, 64, 128, 256):
        mo = hf.make_march_opts(steps=st, far_dist=600.0, stream=stream.cuda_stream)
        mframe = lambda r: hf.hf_render_march(ctx, cams[r % 12:r % 12 + 1],
                                              outs[r % 12:r % 12 + 1], mo)
        mbatch = lambda r: hf.hf_render_march(ctx, cams, outs, mo)
        ev_ms(mframe, 24)
        row = {"frame_ms": ev_ms(mframe, 40), "batch12_ms": ev_ms(mbatch, 10)}
        row["metrics_by_pitch"] = by_pitch()
        res["march_%d" % st] = row
    # the paper's Scattered method at three densities (footprint samples across x
    # along x points per column interval), scored the same way
    fps = synth.footprints(cams, far=600.0)
    for nu, nv, nz in ((512, 512, 8), (1024, 1024, 16), (2048, 2048, 32)):
        so = hf.make_scatter_opts(nu=nu, nv=nv, nz=nz, depth_max=1024.0, stream=stream.cuda_stream)
        sframe = lambda r: hf.hf_render_scatter(ctx, cams[r % 12:r % 12 + 1], outs[r % 12:r % 12 + 1],
                                                fps[r % 12:r % 12 + 1], so)
        sbatch = lambda r: hf.hf_render_scatter(ctx, cams, outs, fps, so)
        ev_ms(sframe, 24)
        row = {"frame_ms": ev_ms(sframe, 40), "batch12_ms": ev_ms(sbatch, 10),
               "footprint_samples": nu * nv, "points_per_column_interval": nz,
               "metrics_by_pitch": by_pitch()}
        res["scatter_%dx%dx%d" % (nu, nv, nz)] = row
    # the paper's voxel-accelerated march (RayVoxel): its publication grid (4, 8, 2), its
    # shipping grid (2, 4, 1), and denser leaf sampling; build and one crater repair timed
    for v, inner in (((4, 8, 2), 4), ((4, 8, 2), 16), ((2, 4, 1), 4)):
        t0 = time.perf_counter()
        hf.hf_voxel_build(ctx, *v)
        build_ms = (time.perf_counter() - t0) * 1e3
        words = 0
        for l in range(16):
            try:
                words += hf.hf_read_voxels(ctx, l).size
            except hf.HFError:
                break
        vo = hf.make_voxel_opts(inner=inner, far_dist=600.0, stream=stream.cuda_stream)
        vframe = lambda r: hf.hf_render_voxel(ctx, cams[r % 12:r % 12 + 1], outs[r % 12:r % 12 + 1], vo)
        vbatch = lambda r: hf.hf_render_voxel(ctx, cams, outs, vo)
        ev_ms(vframe, 24)
        row = {"frame_ms": ev_ms(vframe, 40), "batch12_ms": ev_ms(vbatch, 10),
               "build_ms": build_ms, "occupancy_mib": words * 4 / 2**20, "inner": inner,
               "metrics_by_pitch": by_pitch()}
        # one 64 x 64 crater edit: cells, cell pyramid and voxel pyramid repaired
        x0, y0, blk = synth.crater_edit(cells, 1024, 8192)
        row["edit_ms"] = ev_ms(lambda r: hf.hf_edit(ctx, x0, y0, blk), 1)
        hf.hf_edit(ctx, x0, y0, cells[y0:y0 + blk.shape[0], x0:x0 + blk.shape[1]].copy())  # undo
        res["voxel_%d%d%d_inner%d" % (v + (inner,))] = row
    ck = clocks.stop()
    hf.hf_destroy(ctx)
    line = {"metric": "frame time, paper protocol (12 views, 1280x800): exact cast vs the "
                      "paper's fixed-step march, Scattered method and RayVoxel, with Section 4.2 "
                      "metrics",
            "value": res["exact"]["frame_ms"], "unit": "ms per 1280x800 frame (exact cast)",
            "n_gpus": 1, "steps": 40, "warmup": 24, "higher_is_better": False,
            "vs_baseline": None, "dtype": "i32 (exact) / f32 (march, scatter)", "data": "synthetic",
            "config": {"workload": "2048x16384 grid (seed 4, 30% slabs), 3 views at each pitch "
                                   "0/-30/-60/-90, 1280x800, hfov 75, far 600 (march); "
                                   "steady-state frames, primary rays only"},
            "results": res, "clocks": ck}
    print(json.dumps(line))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    wl = workload(args.workload)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, budget_s=per_step)
    vals, secs = [], []
    last = None
    for i in range(args.steps):
        t0 = time.perf_counter()
        last = cpu_oracle_sample(wl, budget_s=per_step, seed=i + 1)
        secs.append(time.perf_counter() - t0)
        vals.append(last["value"])
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": "primary rays/s (batched, exact two-interval "
            "height-field ray cast)", "value": value, "unit": "primary rays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64",
            "data": "synthetic", "config": {"workload": wl["name"]},
            "cpu_baseline": dict(last, value=value, nproc=os.cpu_count(), cpu_model=cpu_model()),
            "e2e": {"value": value, "unit": "primary rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # default: about 1 s timed on every workload, so the 200 ms clock sampler
    # sees several samples (50 batched-camera steps; many more single-camera ones)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hf", choices=["hf", "reference"])
    ap.add_argument("--workload", default="c3",
                    choices=["c1", "c2", "c3", "c4", "c4pair", "c5", "protocol"])
    ap.add_argument("--serve-requests", type=int, default=2200)
    ap.add_argument("--frames-per-step", type=int, default=100,
                    help="large-world fly-through frames rendered per step (one batch)")
    ap.add_argument("--mip", type=int, default=0xFFFFFFFF)
    ap.add_argument("--tile-w", type=int, default=0)
    ap.add_argument("--tile-h", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the batched workload's resolutions (small profiling cases)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else {"c1": 20000, "c2": 8000}.get(
            args.workload, 50)
    if args.warmup < 3 and args.impl == "hf":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c5":
        run_serve(args)
    elif args.workload == "protocol":
        run_protocol(args)
    else:
        run_hf(args)


if __name__ == "__main__":
    main()
