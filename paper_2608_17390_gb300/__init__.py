"""Python binding of libhf.so: exact two-interval height-field ray casting on GB300.

A thin ctypes layer over the C ABI in include/hf.h, with the same names:
``hf_create``, ``hf_edit``, ``hf_render``, ``hf_render_noalloc``, ``hf_render_march``,
``hf_sync``, ``hf_destroy``,
``hf_camera_from_pose``, ``hf_validate_camera``, ``hf_validate_cells``,
``hf_strerror``, ``hf_info``, ``hf_read_cells``, ``hf_read_pyramid``, ``hf_read_sun_bounds``,
``hf_rebuild``, ``hf_stats``.  It only marshals arguments: every step of the
ray cast runs in the library's CUDA kernels.  PyTorch provides device memory
(output tensors) and streams.

Importing this module loads libhf.so and raises if it is missing (build it
with ``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU
fallback.  Errors from the library raise ``HFError``.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhf.so")

HF_OK = 0
HF_E_INVALID_ARG = -1
HF_E_OUT_OF_BOUNDS = -2
HF_E_OOM = -3
HF_E_CUDA = -4
HF_E_STEP_LIMIT = -5
HF_E_BUSY = -6

HF_FACE_NX, HF_FACE_PX, HF_FACE_NY, HF_FACE_PY, HF_FACE_NZ, HF_FACE_PZ, HF_FACE_INSIDE = range(7)
HF_FACE_ERROR = 254
HF_FACE_MISS = 255

HF_SHADOWS = 1
HF_PLAIN = 2
HF_SYNC = 4
HF_STATS = 8
HF_NOGRAPH = 16
HF_NOWAIT = 32
HF_HOST_OUTPUTS = 64
HF_SCATTER_RAW = 128
HF_HOST_STAGED = 256
HF_MIP_AUTO = 0xFFFFFFFF
HF_MAX_DIM = 16384
HF_MAX_CAMERAS = 4096
HF_NOALLOC_MAX_CAMERAS = 256
HF_CELLS_WORD32 = 0
HF_CELLS_PAIR16 = 1


class HFError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, hf_strerror(code), code))


class hf_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("cells", ctypes.c_void_p), ("row_stride", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p)]


class hf_pair_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("texels", ctypes.c_void_p), ("row_stride", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p)]


class hf_camera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_int64 * 3), ("fwd", ctypes.c_int32 * 3),
                ("right", ctypes.c_int32 * 3), ("up", ctypes.c_int32 * 3),
                ("w", ctypes.c_uint32), ("h", ctypes.c_uint32)]


class hf_outputs(ctypes.Structure):
    _fields_ = [("hit_cell", ctypes.c_void_p), ("layer", ctypes.c_void_p),
                ("face", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("rgba", ctypes.c_void_p), ("shadow", ctypes.c_void_p)]


class hf_render_opts(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_uint32), ("tile_h", ctypes.c_uint32),
                ("mip_start", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("max_steps", ctypes.c_uint32), ("sun", ctypes.c_int32 * 3),
                ("cuda_stream", ctypes.c_void_p)]


class hf_march_opts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("bisections", ctypes.c_uint32),
                ("far_dist", ctypes.c_float), ("tile_w", ctypes.c_uint32),
                ("tile_h", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p)]


class hf_footprint(ctypes.Structure):
    _fields_ = [("s_lo", ctypes.c_float), ("s_hi", ctypes.c_float), ("k_lat", ctypes.c_float),
                ("u_min", ctypes.c_float)]


class hf_scatter_opts(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_uint32), ("nv", ctypes.c_uint32), ("nz", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("depth_max", ctypes.c_float),
                ("sun", ctypes.c_int32 * 3), ("cuda_stream", ctypes.c_void_p)]


class hf_voxel_desc(ctypes.Structure):
    _fields_ = [("vx", ctypes.c_uint32), ("vy", ctypes.c_uint32), ("vz", ctypes.c_uint32),
                ("levels", ctypes.c_uint32)]


class hf_voxel_opts(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_uint32), ("inner", ctypes.c_uint32),
                ("far_dist", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p)]


class hf_info_t(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("levels", ctypes.c_uint32), ("render_slots", ctypes.c_uint32),
                ("cell_bytes", ctypes.c_uint64), ("pyramid_bytes", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("sm_count", ctypes.c_int32), ("cell_format", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class hf_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("arrival", ctypes.c_double), ("cam", hf_camera),
                ("x0", ctypes.c_uint32), ("y0", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("h", ctypes.c_uint32), ("cells", ctypes.c_void_p), ("outs", hf_outputs)]


class hf_request_result(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_double), ("done", ctypes.c_double),
                ("version", ctypes.c_uint32), ("batch", ctypes.c_uint32)]


class hf_serve_opts(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("output_budget", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("tile_w", ctypes.c_uint32), ("tile_h", ctypes.c_uint32),
                ("mip_start", ctypes.c_uint32)]


HF_REQ_RENDER = 0
HF_REQ_EDIT = 1

# numpy view of hf_camera (same layout as the C struct)
CAMERA_DTYPE = np.dtype(
    [("o", "<i8", (3,)), ("f", "<i4", (3,)), ("r", "<i4", (3,)),
     ("u", "<i4", (3,)), ("w", "<u4"), ("h", "<u4")], align=True)
assert CAMERA_DTYPE.itemsize == ctypes.sizeof(hf_camera)

OUTPUT_FIELDS = ("hit_cell", "layer", "face", "depth", "rgba", "shadow")

_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_SIGS = {
    "hf_create": ([ctypes.POINTER(hf_desc), ctypes.POINTER(_P)], ctypes.c_int),
    "hf_create_pairs": ([ctypes.POINTER(hf_pair_desc), ctypes.POINTER(_P)], ctypes.c_int),
    "hf_validate_pairs": ([_P, _U32, _U32, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
                          ctypes.c_int),
    "hf_edit": ([_P, _U32, _U32, _U32, _U32, _P, ctypes.c_size_t], ctypes.c_int),
    "hf_render": ([_P, _P, _U32, _P, ctypes.POINTER(hf_render_opts)], ctypes.c_int),
    "hf_render_noalloc": ([_P, _P, _U32, _P, ctypes.POINTER(hf_render_opts)], ctypes.c_int),
    "hf_render_march": ([_P, _P, _U32, _P, ctypes.POINTER(hf_march_opts)], ctypes.c_int),
    "hf_render_scatter": ([_P, _P, _U32, _P, _P, ctypes.POINTER(hf_scatter_opts)], ctypes.c_int),
    "hf_scatter_footprint": ([_P, ctypes.c_float, ctypes.POINTER(hf_footprint)], ctypes.c_int),
    "hf_voxel_build": ([_P, ctypes.POINTER(hf_voxel_desc)], ctypes.c_int),
    "hf_read_voxels": ([_P, _U32, _P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hf_render_voxel": ([_P, _P, _U32, _P, ctypes.POINTER(hf_voxel_opts)], ctypes.c_int),
    "hf_sync": ([_P], ctypes.c_int),
    "hf_destroy": ([_P], ctypes.c_int),
    "hf_camera_from_pose": ([ctypes.c_double] * 6 + [_U32, _U32, ctypes.POINTER(hf_camera)],
                            ctypes.c_int),
    "hf_validate_camera": ([_U32, _U32, ctypes.POINTER(hf_camera)], ctypes.c_int),
    "hf_validate_cells": ([_P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hf_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "hf_info": ([_P, ctypes.POINTER(hf_info_t)], ctypes.c_int),
    "hf_read_cells": ([_P, _U32, _U32, _U32, _U32, _P, ctypes.c_size_t], ctypes.c_int),
    "hf_read_pyramid": ([_P, _U32, _P], ctypes.c_int),
    "hf_read_sun_bounds": ([_P, _P, _P], ctypes.c_int),
    "hf_rebuild": ([_P], ctypes.c_int),
    "hf_stats": ([_P, _P], ctypes.c_int),
    "hf_serve_replay": ([_P, _P, _U32, ctypes.POINTER(hf_serve_opts), _P], ctypes.c_int),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhf.so is not built (%s); run the package build first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _check(rc, where):
    if rc != HF_OK:
        raise HFError(rc, where)


def hf_strerror(code):
    return lib.hf_strerror(int(code)).decode()


_CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream's handle


def _current_stream():
    """torch's current stream as a cudaStream_t; its default stream (handle 0)
    is passed as cudaStreamLegacy so that the library orders its work on it
    instead of creating a stream of its own."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or _CUDA_STREAM_LEGACY
    except ImportError:
        pass
    return None


def hf_create(cells, stream=None):
    """Create a context from a uint32 [H, W] host array of cell words.

    stream: a cudaStream_t handle (int), or None for torch's current stream.
    Returns the opaque context handle (int)."""
    c = np.ascontiguousarray(cells, dtype=np.uint32)
    if c.ndim != 2:
        raise ValueError("cells must be a 2-D array")
    H, W = c.shape
    d = hf_desc(W, H, c.ctypes.data, W, stream if stream is not None else _current_stream())
    h = _P()
    _check(lib.hf_create(ctypes.byref(d), ctypes.byref(h)), "hf_create")
    return h.value


def hf_create_pairs(texels, stream=None):
    """Create a context from a uint16 [H, W] host array of paired texels (W
    even; the encoding is described in include/hf.h at hf_pair_desc)."""
    t = np.ascontiguousarray(texels, dtype=np.uint16)
    if t.ndim != 2:
        raise ValueError("texels must be a 2-D array")
    H, W = t.shape
    d = hf_pair_desc(W, H, t.ctypes.data, W, stream if stream is not None else _current_stream())
    h = _P()
    _check(lib.hf_create_pairs(ctypes.byref(d), ctypes.byref(h)), "hf_create_pairs")
    return h.value


def hf_validate_pairs(texels):
    """Returns (code, index of the first bad pair's even texel or None)."""
    t = np.ascontiguousarray(texels, dtype=np.uint16)
    if t.ndim != 2:
        raise ValueError("texels must be a 2-D array")
    H, W = t.shape
    bad = ctypes.c_size_t(0)
    rc = lib.hf_validate_pairs(t.ctypes.data if t.size else None, W, H, W, ctypes.byref(bad))
    return rc, (bad.value if rc != HF_OK else None)


def hf_edit(ctx, x0, y0, block):
    """Overwrite the cells of a rectangle at (x0, y0) with a uint32 [h, w] host array."""
    b = np.ascontiguousarray(block, dtype=np.uint32)
    h, w = b.shape
    _check(lib.hf_edit(ctx, int(x0), int(y0), w, h, b.ctypes.data, w), "hf_edit")


def camera_records(cams):
    """A contiguous CAMERA_DTYPE array from records with fields o, f, r, u, w, h."""
    a = np.asarray(cams)
    if a.dtype != CAMERA_DTYPE:
        out = np.zeros(a.shape, CAMERA_DTYPE)
        for k in CAMERA_DTYPE.names:
            out[k] = a[k]
        a = out
    return np.ascontiguousarray(a.reshape(-1))


def _outputs_array(outs):
    arr = (hf_outputs * len(outs))()
    for i, o in enumerate(outs):
        for k in OUTPUT_FIELDS:
            t = o.get(k) if isinstance(o, dict) else getattr(o, k, None)
            setattr(arr[i], k, None if t is None else int(t.data_ptr()))
    return arr


def make_opts(tile_w=0, tile_h=0, mip_start=HF_MIP_AUTO, flags=0, max_steps=0, sun=(0, 0, 0),
              stream=None):
    return hf_render_opts(tile_w, tile_h, mip_start, flags, max_steps,
                          (ctypes.c_int32 * 3)(*sun), stream)


def hf_render(ctx, cams, outs, opts=None):
    """Render camera records into per-camera dicts of device tensors (pinned
    host tensors with HF_HOST_OUTPUTS in opts.flags).

    cams: CAMERA_DTYPE array (or records with the same fields); outs: a list
    of dicts keyed by hit_cell, layer, face, depth, rgba, shadow (missing or
    None entries are not written); opts: an hf_render_opts or None.

    The render is asynchronous on the context's stream (or opts.cuda_stream):
    keep the output tensors alive until it has completed there (hf_sync, or
    an event on that stream).  torch's caching allocator does not see that
    stream, so a tensor freed early could be handed out again while the
    kernel still writes it."""
    recs = camera_records(cams)
    n = len(recs)
    if len(outs) != n:
        raise ValueError("one output set per camera")
    oarr = _outputs_array(outs)
    popts = ctypes.byref(opts) if opts is not None else None
    rc = lib.hf_render(ctx, recs.ctypes.data if n else None, n, oarr, popts)
    _check(rc, "hf_render")


def hf_render_noalloc(ctx, cams, outs, opts=None):
    """hf_render without any allocation in the library (at most
    HF_NOALLOC_MAX_CAMERAS cameras, context stream only; see include/hf.h)."""
    recs = camera_records(cams)
    n = len(recs)
    if len(outs) != n:
        raise ValueError("one output set per camera")
    oarr = _outputs_array(outs)
    popts = ctypes.byref(opts) if opts is not None else None
    _check(lib.hf_render_noalloc(ctx, recs.ctypes.data if n else None, n, oarr, popts),
           "hf_render_noalloc")


def make_scatter_opts(nu=0, nv=0, nz=0, flags=0, depth_max=0.0, sun=(0, 0, 0), stream=None):
    return hf_scatter_opts(nu, nv, nz, flags, depth_max, (ctypes.c_int32 * 3)(*sun), stream)


def hf_scatter_footprint(cam, far_dist=600.0):
    """(s_lo, s_hi, k_lat, u_min) the library chooses for one camera record."""
    rec = camera_records(np.asarray([cam]))
    c = hf_camera.from_buffer_copy(rec.tobytes())
    f = hf_footprint()
    _check(lib.hf_scatter_footprint(ctypes.byref(c), far_dist, ctypes.byref(f)),
           "hf_scatter_footprint")
    return (f.s_lo, f.s_hi, f.k_lat, f.u_min)


def hf_render_scatter(ctx, cams, outs, footprints=None, opts=None):
    """The paper's Scattered method (comparison renderer; see include/hf.h).
    footprints: float32 [n, 4] (s_lo, s_hi, k_lat, u_min) or None for the
    library's; outs need hit_cell (the screen buffer)."""
    recs = camera_records(cams)
    n = len(recs)
    if len(outs) != n:
        raise ValueError("one output set per camera")
    oarr = _outputs_array(outs)
    fp = None
    if footprints is not None:
        fp = np.ascontiguousarray(footprints, dtype=np.float32).reshape(n, 4)
    popts = ctypes.byref(opts) if opts is not None else None
    _check(lib.hf_render_scatter(ctx, recs.ctypes.data if n else None, n,
                                 fp.ctypes.data if fp is not None else None, oarr, popts),
           "hf_render_scatter")


def hf_voxel_build(ctx, vx=4, vy=8, vz=2, levels=0):
    """Build the context's RayVoxel occupancy pyramid (include/hf.h)."""
    d = hf_voxel_desc(vx, vy, vz, levels)
    _check(lib.hf_voxel_build(ctx, ctypes.byref(d)), "hf_voxel_build")


def hf_read_voxels(ctx, level):
    """uint32 words of one voxel level (Morton-coded 8^3 tiles)."""
    n = ctypes.c_size_t(0)
    _check(lib.hf_read_voxels(ctx, level, None, ctypes.byref(n)), "hf_read_voxels")
    out = np.empty(n.value, np.uint32)
    _check(lib.hf_read_voxels(ctx, level, out.ctypes.data, ctypes.byref(n)), "hf_read_voxels")
    return out


def make_voxel_opts(outer=0, inner=0, far_dist=0.0, flags=0, stream=None):
    return hf_voxel_opts(outer, inner, far_dist, flags, stream)


def hf_render_voxel(ctx, cams, outs, opts=None):
    """RayVoxel render (comparison method; see include/hf.h).  Writes hit_cell,
    layer and depth of each output dict."""
    recs = camera_records(cams)
    n = len(recs)
    if len(outs) != n:
        raise ValueError("one output set per camera")
    oarr = _outputs_array(outs)
    popts = ctypes.byref(opts) if opts is not None else None
    _check(lib.hf_render_voxel(ctx, recs.ctypes.data if n else None, n, oarr, popts),
           "hf_render_voxel")


def make_march_opts(steps=0, bisections=0, far_dist=0.0, tile_w=0, tile_h=0, flags=0,
                    stream=None):
    return hf_march_opts(steps, bisections, far_dist, tile_w, tile_h, flags, stream)


def hf_render_march(ctx, cams, outs, opts=None):
    """The paper's fixed-step ray march (comparison method; see include/hf.h).
    Writes hit_cell, layer and depth of each output dict."""
    recs = camera_records(cams)
    n = len(recs)
    if len(outs) != n:
        raise ValueError("one output set per camera")
    oarr = _outputs_array(outs)
    popts = ctypes.byref(opts) if opts is not None else None
    _check(lib.hf_render_march(ctx, recs.ctypes.data if n else None, n, oarr, popts),
           "hf_render_march")


def hf_sync(ctx):
    _check(lib.hf_sync(ctx), "hf_sync")


def hf_destroy(ctx):
    _check(lib.hf_destroy(ctx), "hf_destroy")


def hf_camera_from_pose(x, y, z, yaw_deg, pitch_deg, hfov_deg, w, h):
    """Quantise a pose; returns one CAMERA_DTYPE record."""
    c = hf_camera()
    _check(lib.hf_camera_from_pose(x, y, z, yaw_deg, pitch_deg, hfov_deg, w, h, ctypes.byref(c)),
           "hf_camera_from_pose")
    rec = np.zeros(1, CAMERA_DTYPE)
    ctypes.memmove(rec.ctypes.data, ctypes.byref(c), ctypes.sizeof(c))
    return rec[0]


def hf_validate_camera(grid_w, grid_h, cam):
    rec = camera_records(np.asarray([cam]))
    c = hf_camera.from_buffer_copy(rec.tobytes())
    return lib.hf_validate_camera(grid_w, grid_h, ctypes.byref(c))


def hf_validate_cells(cells):
    """Returns (code, first_bad_index or None)."""
    c = np.ascontiguousarray(cells, dtype=np.uint32).reshape(-1)
    bad = ctypes.c_size_t(0)
    rc = lib.hf_validate_cells(c.ctypes.data if c.size else None, c.size, ctypes.byref(bad))
    return rc, (bad.value if rc != HF_OK else None)


def hf_info(ctx):
    i = hf_info_t()
    _check(lib.hf_info(ctx, ctypes.byref(i)), "hf_info")
    return {k: getattr(i, k) for k, _ in hf_info_t._fields_}


def hf_read_cells(ctx, x0, y0, w, h):
    out = np.empty((h, w), np.uint32)
    _check(lib.hf_read_cells(ctx, x0, y0, w, h, out.ctypes.data, w), "hf_read_cells")
    return out


def hf_read_pyramid(ctx, level):
    info = hf_info(ctx)
    wk = (info["width"] + (1 << level) - 1) >> level
    hk = (info["height"] + (1 << level) - 1) >> level
    out = np.empty((hk, wk), np.uint32)
    _check(lib.hf_read_pyramid(ctx, level, out.ctypes.data), "hf_read_pyramid")
    return out


def hf_read_sun_bounds(ctx):
    """The per-cell shadow bounds last built by a shadowed render:
    (uint32 [H, W] of F | G << 16 in 2^-8 world units, (sun x, y, z))."""
    info = hf_info(ctx)
    out = np.empty((info["height"], info["width"]), np.uint32)
    sun = (ctypes.c_int32 * 3)()
    _check(lib.hf_read_sun_bounds(ctx, out.ctypes.data, sun), "hf_read_sun_bounds")
    return out, tuple(sun)


def hf_rebuild(ctx):
    _check(lib.hf_rebuild(ctx), "hf_rebuild")


def hf_stats(ctx):
    v = (ctypes.c_uint64 * 5)()
    _check(lib.hf_stats(ctx, v), "hf_stats")
    return dict(node_fetches=v[0], cell_fetches=v[1], rays=v[2], shadow_rays=v[3],
                shadow_fetches=v[4])


def hf_serve_replay(ctx, records, lanes=8, max_batch=8, output_budget=4 << 30, flags=0,
                    tile_w=0, tile_h=0, mip_start=HF_MIP_AUTO, outputs=None):
    """Run a request stream through the library's native serving loop.
    `records` are dicts with "kind" ("render" or "edit"), "arrival" (seconds
    from the start, non-decreasing), "cam" (a camera record, renders) and
    "edit" ((x0, y0, cells), edits).  `outputs`, optional, gives per record a
    dict of device tensors for a render's image (None: the loop's own pool,
    image dropped).  Returns a numpy structured array of (admitted, done,
    version, batch), one row per record."""
    n = len(records)
    if outputs is not None and len(outputs) != n:
        raise ValueError("one output entry (or None) per record")
    reqs = (hf_request * n)()
    keep = []  # the edit cells stay alive through the call
    for i, rec in enumerate(records):
        q = reqs[i]
        q.arrival = float(rec["arrival"])
        if rec["kind"] == "edit":
            x0, y0, blk = rec["edit"]
            blk = np.ascontiguousarray(blk, dtype=np.uint32)
            keep.append(blk)
            q.kind = HF_REQ_EDIT
            q.x0, q.y0, q.h, q.w = int(x0), int(y0), blk.shape[0], blk.shape[1]
            q.cells = blk.ctypes.data
        else:
            q.kind = HF_REQ_RENDER
            c = camera_records(np.array([rec["cam"]]))
            ctypes.memmove(ctypes.addressof(q.cam), c.ctypes.data, ctypes.sizeof(hf_camera))
            if outputs is not None and outputs[i] is not None:
                q.outs = _outputs_array([outputs[i]])[0]
    res = (hf_request_result * n)()
    opts = hf_serve_opts(lanes, max_batch, output_budget, flags, tile_w, tile_h, mip_start)
    _check(lib.hf_serve_replay(ctx, ctypes.cast(reqs, _P) if n else None, n, ctypes.byref(opts),
                               ctypes.cast(res, _P) if n else None), "hf_serve_replay")
    out = np.zeros(n, dtype=[("admitted", "f8"), ("done", "f8"), ("version", "u4"), ("batch", "u4")])
    for i in range(n):
        out[i] = (res[i].admitted, res[i].done, res[i].version, res[i].batch)
    return out


def alloc_outputs(cams, device="cuda", shadows=False, fields=OUTPUT_FIELDS):
    """Allocate one dict of tensors per camera (torch): on `device`, or in
    pinned host memory when device is "pinned" (for HF_HOST_OUTPUTS and
    HF_HOST_STAGED).  Each field is one allocation for all cameras, and a
    camera's tensor is a view of its slice, so consecutive cameras' buffers
    are adjacent (the staged host path then copies a chunk's field at once)."""
    import torch
    dt = dict(hit_cell=torch.int32, layer=torch.uint8, face=torch.uint8, depth=torch.float32,
              rgba=torch.int32, shadow=torch.uint8)
    sizes = [int(c["w"]) * int(c["h"]) for c in camera_records(cams)]
    total = sum(sizes)
    outs = [{} for _ in sizes]
    for k in fields:
        if k == "shadow" and not shadows:
            continue
        if device == "pinned":
            block = torch.empty(total, dtype=dt[k], pin_memory=True)
        else:
            block = torch.empty(total, dtype=dt[k], device=device)
        start = 0
        for o, n in zip(outs, sizes):
            o[k] = block[start:start + n]
            start += n
    return outs
