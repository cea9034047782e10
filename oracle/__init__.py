"""CPU oracle for the two-interval height-field ray cast.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library and its binding) never imports this package, and this package never
imports the product.

Two independent implementations live here:
  * ``hf_oracle.c`` (loaded through ctypes): the plain definition stepped cell
    by cell, exact integer predicates, FP64 depth and colour;
  * ``brute.py``: a pure-Python checker with exact fractions that builds each
    cell's visit interval straight from the definition (tiny grids only).
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

S = 65536
# Direction toward the sun: elevation 30 deg, azimuth 135 deg (clockwise from
# +y), scaled to length 2**19 and rounded once.
DEFAULT_SUN = (321060, -321060, 262144)

FACE_NX, FACE_PX, FACE_NY, FACE_PY, FACE_NZ, FACE_PZ, FACE_INSIDE = range(7)
FACE_MISS = 255
MISS_CELL = 0xFFFFFFFF


def build(force=False):
    """Compile hf_oracle.c into liboracle.so next to it (gcc, no CUDA)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("HF_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_render.argtypes = [P, I64, I64, P, P, ctypes.c_int, I64, P,
                                      P, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_render.restype = ctypes.c_int
        lib.oracle_trace_rays.argtypes = [P, I64, I64, I64, P, P, P, ctypes.c_int,
                                          P, P, P, P, P, P, P]
        lib.oracle_trace_rays.restype = ctypes.c_int
        lib.oracle_pyramid.argtypes = [P, I64, I64, ctypes.c_int, P]
        lib.oracle_pyramid.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _outputs(n, shadows):
    return dict(
        hit_cell=np.empty(n, np.uint32), layer=np.empty(n, np.uint8),
        face=np.empty(n, np.uint8), depth=np.empty(n, np.float64),
        rgba=np.empty(n, np.uint32),
        shadow=np.zeros(n, np.uint8) if shadows else None,
        steps=np.empty(n, np.int64),
    )


def cam_params(cam):
    """14 int64 camera parameters (origin, F, R, U, w, h) from a camera record."""
    return np.array(list(cam["o"]) + list(cam["f"]) + list(cam["r"]) + list(cam["u"])
                    + [int(cam["w"]), int(cam["h"])], dtype=np.int64)


def render(cells, cam, shadows=False, sun=DEFAULT_SUN, pix=None, nthreads=1):
    """Oracle render of one camera record; returns a dict of flat arrays.

    pix: optional array of pixel indices py*w+px; outputs follow its order.
    """
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    H, W = cells.shape
    p = cam_params(cam)
    n = int(p[12] * p[13]) if pix is None else len(pix)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.uint32)
    L = np.array(sun, dtype=np.int64)
    out = _outputs(n, shadows)
    _load().oracle_render(_ptr(cells), W, H, _ptr(p), _ptr(L), int(bool(shadows)), n,
                          _ptr(pixa), _ptr(out["hit_cell"]), _ptr(out["layer"]),
                          _ptr(out["face"]), _ptr(out["depth"]), _ptr(out["rgba"]),
                          _ptr(out["shadow"]), _ptr(out["steps"]), int(nthreads))
    return out


def trace_rays(cells, o, d, shadows=False, sun=DEFAULT_SUN):
    """Oracle trace of explicit rays: o, d are int64 arrays of shape (n, 3)."""
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    H, W = cells.shape
    o = np.ascontiguousarray(o, dtype=np.int64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.int64).reshape(-1, 3)
    n = o.shape[0]
    L = np.array(sun, dtype=np.int64)
    out = _outputs(n, shadows)
    _load().oracle_trace_rays(_ptr(cells), W, H, n, _ptr(o), _ptr(d), _ptr(L),
                              int(bool(shadows)), _ptr(out["hit_cell"]), _ptr(out["layer"]),
                              _ptr(out["face"]), _ptr(out["depth"]), _ptr(out["rgba"]),
                              _ptr(out["shadow"]), _ptr(out["steps"]))
    return out


def levels_for(W, H):
    """Number of pyramid levels above the cells: ceil(log2(max(W, H)))."""
    m = max(W, H)
    L = 0
    while (1 << L) < m:
        L += 1
    return L


def pyramid(cells):
    """Oracle min/max pyramid: list of uint32 arrays, level 1 .. L."""
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    H, W = cells.shape
    L = levels_for(W, H)
    shapes = [((H + (1 << k) - 1) >> k, (W + (1 << k) - 1) >> k) for k in range(1, L + 1)]
    total = sum(a * b for a, b in shapes)
    out = np.zeros(max(total, 1), dtype=np.uint32)
    _load().oracle_pyramid(_ptr(cells), W, H, L, _ptr(out))
    levels, off = [], 0
    for (hk, wk) in shapes:
        levels.append(out[off:off + hk * wk].reshape(hk, wk))
        off += hk * wk
    return levels


def ray_dirs(cam):
    """Integer per-pixel ray directions of a camera record, shape (h*w, 3)."""
    w, h = int(cam["w"]), int(cam["h"])
    py, px = np.mgrid[0:h, 0:w]
    a = (2 * px + 1 - w).reshape(-1, 1).astype(np.int64)
    b = (h - 1 - 2 * py).reshape(-1, 1).astype(np.int64)
    F = np.array(cam["f"], np.int64)
    R = np.array(cam["r"], np.int64)
    U = np.array(cam["u"], np.int64)
    return F[None, :] + a * R[None, :] + b * U[None, :]
