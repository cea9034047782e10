"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds no part of the ray-casting method: it only draws terrain
grids, camera poses, integer camera records and crater edits from fixed seeds.
Both the CPU oracle (``oracle/``) and the CUDA library consume what it
returns; neither imports the other.

Cell word layout (uint32, little-endian bytes): byte0 = h0 (floor top),
byte1 = h1 (slab underside), byte2 = h2 (slab top), byte3 = material.
A cell has a slab iff h1 > h0 (and then h2 >= h1); a cell without a slab
stores h1 = h2 = 0.  This is the two-interval ground sample of the paper's
data section (floor, cave ceiling, slab top), re-encoded as one 32-bit word.

Random numbers come from a counter-based generator: every draw is a pure
function of (seed, stream, index), so any subset of a grid can be regenerated
independently and in any order.
"""

from .rng import mix64, unit_float, uniform_int
from .terrain import (
    value_noise,
    make_grid,
    pack_cells,
    unpack_cells,
    grid_hash,
    crater_edit,
)
from .pairs import pairify, encode_pairs
from .scatter import footprint_for, footprints
from .cameras import (
    CAMERA_DTYPE,
    pose_to_camera,
    ray_camera,
    camera_array,
    config_c1,
    config_c2,
    config_c3,
    c3_cameras,
    config_c4,
    config_c4_frames,
    small_c2,
    protocol_cameras,
    PROTOCOL_PITCHES,
)

from .requests import poisson_requests, SERVING_RESOLUTIONS

__all__ = [
    "mix64", "unit_float", "uniform_int",
    "value_noise", "make_grid", "pack_cells", "unpack_cells", "grid_hash",
    "crater_edit",
    "CAMERA_DTYPE", "pose_to_camera", "ray_camera", "camera_array",
    "config_c1", "config_c2", "config_c3", "c3_cameras", "config_c4", "config_c4_frames",
    "small_c2", "poisson_requests", "SERVING_RESOLUTIONS", "protocol_cameras",
    "PROTOCOL_PITCHES",
]
