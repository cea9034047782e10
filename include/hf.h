/*
 * hf.h -- C ABI of an exact two-interval height-field ray caster (GB300, sm_103a).
 *
 * The operation (arxiv 2608.17390, Malyshau, "Six Ways to Draw Vangers with
 * WebGPU"): each ground cell holds two solid intervals, a floor [.., h0] and an
 * optional slab [h1, h2] (Section 2, The Data); a point is solid when
 * z <= h0 or h1 <= z <= h2 (the SOLID predicate of Section 3.1, closed ends,
 * no lower bound on the floor); one ray is cast per pixel and the first solid
 * point along it is reported; a bounded rectangular edit must be visible on the
 * next render without a rebuild (Sections 2 and 4.4).  The library answers
 * this exactly with fixed-point integer arithmetic, skipping empty space with a
 * conservative min/max pyramid (the hierarchy of Section 3.2 may pass over a
 * region only when it is known to hold nothing) that an edit repairs
 * incrementally.
 *
 * Units.  One world unit is one cell width and one height step.  Positions are
 * fixed point in units of 2^-16 world units.  A pixel ray is p(t) = O + t d,
 * t >= 0, with integer O and d.
 *
 * Cell word (uint32, little-endian bytes): byte0 h0, byte1 h1, byte2 h2,
 * byte3 material.  A cell has a slab iff h1 > h0, and then h2 >= h1; a cell
 * without a slab must store h1 = h2 = 0.  Other combinations are rejected.
 *
 * Result of a ray.  The ray visits the cells whose (half-open) column it
 * occupies for a positive length of t; each visit covers a closed interval of
 * t.  The hit is the first visited cell, in visit order, whose closed interval
 * holds a solid t, at the smallest such t; the ray misses when it leaves the
 * grid first.  At an exact cell corner the ray steps diagonally; the entry
 * face is then the X face.
 *
 * Errors.  Every function returns an int: HF_OK (0) or a negative HF_E_* code.
 * No C++ exception crosses this interface.  A context is not thread-safe: use
 * one context per host thread or lock around calls.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define HF_OK 0
#define HF_E_INVALID_ARG (-1)   /* null pointer, zero or oversize extent, invalid cell, bad camera */
#define HF_E_OUT_OF_BOUNDS (-2) /* edit/read rectangle outside the grid */
#define HF_E_OOM (-3)           /* device or pinned host allocation failed */
#define HF_E_CUDA (-4)          /* a CUDA runtime call failed */
#define HF_E_STEP_LIMIT (-5)    /* a ray exceeded its traversal step guard (its face = HF_FACE_ERROR) */
#define HF_E_BUSY (-6)          /* every render slot is in flight (only with HF_NOWAIT) */

/* face codes written to hf_outputs.face */
#define HF_FACE_NX 0     /* entered through its -X side (ray moving +x) */
#define HF_FACE_PX 1     /* entered through its +X side (ray moving -x) */
#define HF_FACE_NY 2     /* entered through its -Y side (ray moving +y) */
#define HF_FACE_PY 3     /* entered through its +Y side (ray moving -y) */
#define HF_FACE_NZ 4     /* slab underside (cave ceiling), ray moving up */
#define HF_FACE_PZ 5     /* top of the floor or of the slab, ray moving down */
#define HF_FACE_INSIDE 6 /* the ray starts inside solid (t = 0) */
#define HF_FACE_ERROR 254
#define HF_FACE_MISS 255

/* hf_render_opts.flags */
#define HF_SHADOWS 1u /* trace one shadow ray per hit toward the sun */
#define HF_PLAIN 2u   /* one non-persistent launch per camera instead of one batched launch
                         (always so for a single camera, unless HF_NOGRAPH asks for the
                         persistent kernel) */
#define HF_SYNC 4u    /* wait for the render and return its status (HF_E_STEP_LIMIT) */
#define HF_STATS 8u   /* count node and cell fetches (read back with hf_stats) */
#define HF_NOGRAPH 16u /* launch directly instead of replaying a captured CUDA graph */
#define HF_NOWAIT 32u /* return HF_E_BUSY instead of waiting for a free render slot */
#define HF_SCATTER_RAW 128u /* hf_render_scatter: leave the packed words in hit_cell, no resolve */
#define HF_HOST_STAGED 256u /* the output buffers are pinned HOST memory: the library renders
                               the batch in chunks of equal pixel counts (at least 2^19
                               pixels; cameras split into row bands, each rendered as a camera
                               of its own with the same pixel rays) into its own device staging (four buffers of the
                               largest chunk, allocated on first use) and copies each finished
                               chunk back on a copy stream while later chunks render; bands
                               whose host buffers of one field lie back to back share one
                               copy (hf_render only; not with HF_HOST_OUTPUTS, HF_PLAIN or
                               HF_NOWAIT) */
#define HF_HOST_OUTPUTS 64u /* the output buffers are pinned HOST memory (cudaHostAlloc or
                               cudaHostRegister): the kernel writes the results there itself,
                               over the host link, with no separate copy (hf_render only) */

#define HF_MIP_AUTO 0xFFFFFFFFu

#define HF_MAX_DIM 16384u     /* largest grid width/height and image width/height */
#define HF_MAX_CAMERAS 4096u  /* largest batch in one hf_render call */

/* hf_info_t.cell_format: how the device stores the cells (level 0) */
#define HF_CELLS_WORD32 0u /* one 4-byte word per cell (hf_create) */
#define HF_CELLS_PAIR16 1u /* one 2-byte texel per cell, paired (hf_create_pairs) */

/* --------------------------------------------------------------- types */
typedef struct hf_ctx hf_ctx; /* opaque: owns the device grid, pyramid and scratch */

typedef struct {
    uint32_t width, height; /* grid size in cells, 1..HF_MAX_DIM each */
    const uint32_t *cells;  /* HOST pointer to height rows of row_stride cell words */
    size_t row_stride;      /* cells per row in `cells`; 0 means width */
    void *cuda_stream;      /* cudaStream_t all work of this context is ordered on;
                               NULL: the library creates (and destroys) its own */
} hf_desc;

/* A world in the paired-texel encoding of the paper's data section (Section 2,
 * The Data: a double-level region stores, per texel PAIR, the floor top in the
 * even texel, the slab top in the odd texel, and the cave ceiling as delta bits
 * in both).  The paper gives no bit layout; this library's is:
 *   texel = uint16: low byte altitude v, high byte meta m;
 *   m bit 7 = the pair (x even, x + 1) is double-level (equal on both texels),
 *   m bits 6..3 = a delta nibble, m bits 2..0 = material (0..7).
 *   Single-level pair: each texel is a cell with h0 = v, no slab; both nibbles 0.
 *   Double-level pair: both cells have h0 = v(even), h2 = v(odd),
 *   h1 = h2 - (16 * nibble(even) + nibble(odd)), needing h0 < h1 <= h2, and the
 *   material of their own texel.
 * The device keeps 2 bytes per cell (half of hf_create's) and decodes in the
 * kernels; every result equals that of hf_create on the decoded cells. */
typedef struct {
    uint32_t width, height;  /* grid size in cells; width even, 2..HF_MAX_DIM */
    const uint16_t *texels;  /* HOST pointer to height rows of row_stride texels */
    size_t row_stride;       /* texels per row; 0 means width */
    void *cuda_stream;       /* as in hf_desc */
} hf_pair_desc;

/* Integer camera.  Pixel (px, py), py = 0 at the top row, looks along
 *   d = fwd + (2 px + 1 - w) right + (h - 1 - 2 py) up.
 * Valid when 0 <= origin[0] < W*65536, 0 <= origin[1] < H*65536,
 * 0 <= origin[2] < 2^28, 1 <= w, h <= HF_MAX_DIM, and |fwd_i|, |right_i|*(w-1),
 * |up_i|*(h-1) and every corner pixel's |d_i| are each below 2^21. */
typedef struct {
    int64_t origin[3]; /* 2^-16 world units */
    int32_t fwd[3], right[3], up[3];
    uint32_t w, h;
} hf_camera;

/* Per-camera output buffers, each w*h elements in row-major pixel order
 * (py*w + px): DEVICE memory, or pinned HOST memory with HF_HOST_OUTPUTS.
 * (HF_HOST_STAGED: pinned HOST memory too).  Caller-owned; they must stay
 * allocated until the render has completed on its stream.  A NULL member is
 * not written. */
typedef struct {
    uint32_t *hit_cell; /* y*W + x of the hit cell; 0xFFFFFFFF on a miss */
    uint8_t *layer;     /* 0 floor, 1 slab, 255 miss */
    uint8_t *face;      /* HF_FACE_* */
    float *depth;       /* t*|d|/65536 world units (Euclidean); +inf on a miss */
    uint32_t *rgba;     /* shaded colour, bytes r,g,b,a */
    uint8_t *shadow;    /* 1 when the sun is occluded (written only with HF_SHADOWS) */
} hf_outputs;

typedef struct {
    uint32_t tile_w, tile_h; /* pixels per warp tile (powers of two, product 32..256);
                                0,0 = default 8 x 4 */
    uint32_t mip_start;      /* coarsest pyramid level the traversal uses and starts at;
                                0 = flat cell-by-cell DDA; HF_MIP_AUTO = library default;
                                larger values are clamped to the pyramid's top level */
    uint32_t flags;          /* HF_SHADOWS | HF_PLAIN | HF_SYNC | HF_STATS | HF_NOGRAPH | HF_NOWAIT
                                | HF_HOST_OUTPUTS | HF_HOST_STAGED */
    uint32_t max_steps;      /* traversal iterations allowed per ray; 0 = default guard */
    int32_t sun[3];          /* direction toward the sun; all zero = (321060, -321060, 262144),
                                elevation 30 deg, azimuth 135 deg; each |sun_i| < 2^21.
                                With HF_SHADOWS and a sun that rises (sun[2] > 0), is not
                                vertical, and clears the 255-unit height range within
                                1024 cells, the first such render builds per-cell shadow
                                bounds for this sun (4 bytes per cell, allocated then,
                                rebuilt when a render asks for another sun, repaired by
                                hf_edit): a shadow ray whose origin they decide is not
                                traced; the shadow bit is the same either way. */
    void *cuda_stream;       /* stream for this render; NULL = the context's stream */
} hf_render_opts;

typedef struct {
    uint32_t width, height, levels; /* grid size; pyramid levels above the cells */
    uint32_t render_slots;          /* concurrent renders the context can hold in flight */
    uint64_t cell_bytes;            /* device bytes of the cell grid */
    uint64_t pyramid_bytes;         /* device bytes of the pyramid (levels 1..levels) */
    uint64_t scratch_bytes;         /* device bytes of per-render scratch (camera tables) */
    int32_t device;                 /* CUDA device ordinal */
    int32_t sm_count;
    uint32_t cell_format;           /* HF_CELLS_WORD32 or HF_CELLS_PAIR16 */
    uint32_t reserved;
} hf_info_t;

/* ------------------------------------------------------------ functions */

/* Create a context: validates every cell (Section 2 two-interval encoding),
 * copies the grid to the device, builds the pyramid (levels 1..ceil(log2
 * max(W,H))).  The caller may free desc->cells when this returns.  The device
 * is the current CUDA device.  On error *out is set to NULL.
 * Errors: HF_E_INVALID_ARG (null, bad size, invalid cell), HF_E_OOM, HF_E_CUDA. */
int hf_create(const hf_desc *desc, hf_ctx **out);

/* hf_create for a paired-texel world (hf_pair_desc).  The caller may free
 * desc->texels when this returns.  Errors: HF_E_INVALID_ARG (null, bad or odd
 * width, a pair that breaks the encoding's rules), HF_E_OOM, HF_E_CUDA. */
int hf_create_pairs(const hf_pair_desc *desc, hf_ctx **out);

/* Overwrite the cells of rectangle [x0, x0+w) x [y0, y0+h) with `cells` (HOST
 * pointer, h rows of row_stride cells; 0 = w) and repair the pyramid nodes that
 * cover it, level by level (the incremental rebuild of affected cells and their
 * ancestors, Sections 2 and 3.2).  The cells are staged before return, so the
 * caller may reuse its buffer at once.  The edit is ordered on the context's
 * stream after every render issued before it (renders issued on other streams
 * included) and before every render issued after it: those renders see it,
 * earlier ones do not (the first-frame visibility of Section 4.4).
 * For a paired-texel world (hf_create_pairs) the cells are still cell words:
 * x0 and w must be even, and each pair must be representable (no slab in
 * either cell, or the same slab column in both, materials 0..7); the library
 * encodes them.  w = 0 or h = 0 is a no-op.
 * Errors: HF_E_INVALID_ARG (null, invalid or unrepresentable cell, odd x0 or w
 * in a paired-texel world),
 * HF_E_OUT_OF_BOUNDS (rectangle outside the grid), HF_E_OOM, HF_E_CUDA. */
int hf_edit(hf_ctx *ctx, uint32_t x0, uint32_t y0, uint32_t w, uint32_t h,
            const uint32_t *cells, size_t row_stride);

/* Render n cameras (HOST array) into outs[0..n-1]: per pixel, the first solid
 * point of its ray under the SOLID predicate of Section 3.1 (closed ends, the
 * floor unbounded below), the exact result of the flat per-cell CPU ray cast
 * the paper evaluates its renderers against (Section 4.1); misses keep the
 * cleared far values rather than a made-up ground hit (Section 3.1).  The hit
 * record layout is given at hf_outputs; shading and the optional shadow ray
 * at hf_render_opts.  outs is a HOST array of structs that
 * hold DEVICE pointers, or pinned HOST pointers with HF_HOST_OUTPUTS: each
 * non-NULL one is then checked with cudaPointerGetAttributes and replaced by
 * its device alias; the results are in host memory once the render's stream
 * has completed).  Asynchronous on the render stream unless HF_SYNC.
 * opts = NULL uses the defaults.  n = 0 is a no-op.
 * Errors: HF_E_INVALID_ARG (null, n > HF_MAX_CAMERAS, invalid camera or tile
 * shape, with HF_HOST_OUTPUTS an output pointer that is neither device memory
 * nor mapped pinned host memory), HF_E_BUSY (HF_NOWAIT and no free slot),
 * HF_E_CUDA, and with HF_SYNC HF_E_STEP_LIMIT when a ray hit its step guard. */
int hf_render(hf_ctx *ctx, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
              const hf_render_opts *opts);

/* Allocation-free variant of hf_render.  The paper has no counterpart; it is
 * here for callers that must not allocate device memory while they run: a
 * render loop whose GPU memory budget is fixed at start-up, or a
 * latency-critical thread where cudaMalloc/cudaFree could stall or implicitly
 * synchronise the device.  hf_render may allocate (per-slot camera tables,
 * pinned staging, CUDA graphs) on its first calls or when a batch grows; this
 * function calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * It renders n <= HF_NOALLOC_MAX_CAMERAS cameras with the same kernel and the
 * same results as hf_render, always as one batched launch on the context's
 * own stream (opts->cuda_stream must be NULL or that stream), so edits and
 * renders stay ordered.  Accepted flags: HF_SHADOWS and HF_SYNC (with HF_SYNC
 * the step-guard status is returned; without it this entry point reports no
 * step-guard status, and hf_sync does not see it).  Any other flag is refused
 * with HF_E_INVALID_ARG before anything is enqueued.
 *
 * Scratch: one statically allocated device array of about 28 KiB (batch
 * header with the tile counter, camera table, status word) that every GPU
 * loading this library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) once.
 * All calls share the array and it keeps the last call's contents; each
 * call rewrites what must start at zero.  Calls whose GPU work overlaps
 * (from several threads or contexts on one device) race on the array; calls
 * ordered on one stream do not.  The camera table is copied from pageable
 * host memory, so the call waits for earlier work on the context's stream
 * before returning.
 * Errors: HF_E_INVALID_ARG (null, n > HF_NOALLOC_MAX_CAMERAS, invalid camera,
 * tile shape, stream or flag), HF_E_CUDA, and with HF_SYNC HF_E_STEP_LIMIT. */
#define HF_NOALLOC_MAX_CAMERAS 256u
int hf_render_noalloc(hf_ctx *ctx, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                      const hf_render_opts *opts);

/* Options of the fixed-step comparison marcher. */
typedef struct {
    uint32_t steps;          /* forward samples over the clipped segment; 0 = 128 */
    uint32_t bisections;     /* bisection iterations after the first solid sample; 0 = 4 */
    float far_dist;          /* far plane distance in world units; 0 = 600 */
    uint32_t tile_w, tile_h; /* warp tile as in hf_render_opts; 0,0 = 8 x 4 */
    uint32_t flags;          /* HF_SYNC */
    void *cuda_stream;       /* NULL = the context's stream */
} hf_march_opts;

/* The paper's Scattered method (Section 3: its object-order painter recast as a
 * parallel atomic scatter), as a comparison renderer.  Per camera, an nu x nv
 * grid of samples covers a camera-aligned ground footprint: longitudinal s
 * along the horizontal direction 90 degrees left of the camera's right vector,
 * s = s_lo + (s_hi - s_lo) t^2 with t = (j + 0.5) / nv (samples crowd near the
 * camera end), lateral u along the right vector, |u| <= u_min + k_lat |s| (a
 * trapezoid, like a pitched camera's view of the ground).
 * Each sample walks its cell's column (nz points from the floor top down to 0,
 * and for a slab nz points from its top down to its underside), projects every
 * point with the camera (d = F + aR + bU, pixel (floor((a + w)/2), floor((h -
 * b)/2)), points behind or outside dropped) and keeps per pixel, with a 32-bit
 * atomicMin, the least (24-bit quantised Euclidean depth << 8 | material |
 * layer << 3).  The resolve writes depth, the cell under the reconstructed
 * point, layer, face +Z and the material's colour lit from above; pixels no
 * point reached are misses.  float32 arithmetic in a fixed order: results are
 * reproducible bit for bit.  Approximate by design (gaps where the footprint is
 * sparse; the paper's coherence metric measures them). */
typedef struct {
    float s_lo, s_hi; /* longitudinal range (world units), s_hi > s_lo */
    float k_lat;      /* growth of the lateral half-width per unit of |s| */
    float u_min;      /* lateral half-width at s = 0 */
} hf_footprint;

typedef struct {
    uint32_t nu, nv;    /* footprint samples across and along (<= 8192 each); 0 = 1024 */
    uint32_t nz;        /* points per column interval (2..4096); 0 = 16 */
    uint32_t flags;     /* HF_SYNC | HF_SCATTER_RAW */
    float depth_max;    /* depth quantisation range, world units (2^24 steps); 0 = 1024 */
    int32_t sun[3];     /* as in hf_render_opts */
    void *cuda_stream;  /* NULL = the context's stream */
} hf_scatter_opts;

/* A footprint that bounds what the camera can see: a 5 x 5 grid of image rays
 * followed to the plane z = 0 or to far_dist; the s range bounds their ground
 * points; k_lat is the growth of the widest |u| from the image's bottom row of
 * points to its top row per unit of s (0 if it shrinks); u_min is then the
 * least value that holds every point; 5 % margins.  Host only.
 * Errors: HF_E_INVALID_ARG (null, far_dist <= 0, a right vector with no
 * horizontal part). */
int hf_scatter_footprint(const hf_camera *cam, float far_dist, hf_footprint *out);

/* Scatter-render n cameras into outs (DEVICE buffers; hit_cell is required: it
 * is the screen buffer the atomics target, then the resolved cell index).
 * fps: n footprints (HOST), or NULL for hf_scatter_footprint(cam, 600).
 * Asynchronous on the render stream unless HF_SYNC; ordered after edits like
 * hf_render.  Errors: HF_E_INVALID_ARG (null, n > HF_MAX_CAMERAS, invalid
 * camera or footprint, missing hit_cell, bad densities), HF_E_CUDA. */
int hf_render_scatter(hf_ctx *ctx, const hf_camera *cams, uint32_t n, const hf_footprint *fps,
                      const hf_outputs *outs, const hf_scatter_opts *opts);

/* The paper's voxel-accelerated ray march, RayVoxel (Section 3), as a
 * comparison renderer.  A conservative occupancy pyramid: level-0 voxel
 * (i, j, k) covers cells [i vx, (i+1) vx) x [j vy, (j+1) vy) and heights
 * [k vz, (k+1) vz] (closed) and is occupied when some of its cells is solid at
 * some of its heights; each higher level is the union of eight children; every
 * level is stored as Morton-coded 8 x 8 x 8 tiles of bits (tile (tx, ty, tz) at
 * (tz TY + ty) TX + tx, 16 words per tile, voxel bit at the interleaving of
 * the bits of x, y, z from the lowest).  The paper's publication grid (4,8,2)
 * of its 2048 x 16384 level is vx 4, vy 8, vz 2 (18.29 MiB).  Traversal per
 * pixel ray (float32 in a fixed order, no fused multiply-add): clip to the
 * voxel box and the far distance, start at the top level, advance an empty
 * voxel to its exit plane (climbing when the plane bounds the parent), open an
 * occupied one, and sample an occupied leaf at `inner` midpoints of the ray's
 * stretch in it; the first solid sample is the hit.  A feature thinner than
 * the sample spacing can be missed (the paper's trade-off). */
typedef struct {
    uint32_t vx, vy, vz;  /* voxel extent in cells and height units (1..64, 1..64, 1..256) */
    uint32_t levels;      /* pyramid levels (1..16); 0 = until the top level has at most 8
                             voxels along every axis */
} hf_voxel_desc;

typedef struct {
    uint32_t outer;     /* traversal steps per ray (<= 2^20); 0 = 1024 */
    uint32_t inner;     /* samples per occupied leaf voxel (<= 4096); 0 = 4 */
    float far_dist;     /* world units; 0 = 600 */
    uint32_t flags;     /* HF_SYNC */
    void *cuda_stream;  /* NULL = the context's stream */
} hf_voxel_opts;

/* Build (or rebuild with new extents) the context's voxel pyramid from its
 * cells; later hf_edit and hf_rebuild calls keep it current (the edited
 * columns' voxels at level 0, then the covering words of each level above).
 * Synchronous.  Errors: HF_E_INVALID_ARG (null, extents or levels out of
 * range), HF_E_OOM, HF_E_CUDA. */
int hf_voxel_build(hf_ctx *ctx, const hf_voxel_desc *desc);

/* Copy voxel level `level` to HOST memory (synchronous): with out == NULL,
 * store its word count in *n_words; else *n_words must equal that count.
 * Errors: HF_E_INVALID_ARG (no voxel pyramid, bad level or count), HF_E_CUDA. */
int hf_read_voxels(hf_ctx *ctx, uint32_t level, uint32_t *out, size_t *n_words);

/* RayVoxel-render n cameras: writes hit_cell, layer and depth (a miss: 0xFFFFFFFF,
 * 255, +inf); face, rgba, shadow are not written.  Needs hf_voxel_build first.
 * Ordering as hf_render.  Errors: as hf_render, and HF_E_INVALID_ARG without a
 * voxel pyramid or with out-of-range options. */
int hf_render_voxel(hf_ctx *ctx, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                    const hf_voxel_opts *opts);

/* The paper's own height-field ray march (Section 3.1), for comparison with
 * the exact cast: per pixel ray, clip the segment at the far distance and, for
 * a descending ray, at z = 0; take `steps` samples spaced uniformly over it
 * (the paper's text; its listing's loop would space them geometrically); stop
 * at the first sample inside a solid interval of the cell holding it; refine
 * with `bisections` halvings.  float32 arithmetic in a fixed order, no fused
 * multiply-add.  It can step over features thinner than its sample spacing.
 * Writes hit_cell, layer and depth (face, rgba, shadow are not written); a ray
 * with no solid sample misses (0xFFFFFFFF, 255, +inf).  Same ordering rules as
 * hf_render.  Errors: as hf_render (steps or bisections above 65536, or a
 * non-positive far distance, are HF_E_INVALID_ARG). */
int hf_render_march(hf_ctx *ctx, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                    const hf_march_opts *opts);

/* Wait for all work the context issued (every render slot and the context
 * stream).  Returns HF_E_STEP_LIMIT if any ray of any render since the last
 * hf_sync hit its step guard (and clears that flag), else HF_OK / HF_E_CUDA. */
int hf_sync(hf_ctx *ctx);

/* The end of a context's life (the paper has no counterpart: its renderers
 * release their GPU resources with the graphics device).  Synchronise, then
 * free every device and host resource of the context.  NULL is accepted.
 * Returns HF_OK or HF_E_CUDA. */
int hf_destroy(hf_ctx *ctx);

/* Host helper: quantise a pose into an integer camera, in float64.  yaw 0
 * looks along +y, yaw 90 along +x; pitch < 0 looks down; hfov is the
 * horizontal field of view with square pixels.  The focal length is fixed in
 * pixels, f = (w/2)/tan(hfov/2), independent of h (Section 4.1 records a
 * reference camera whose focal length scaled with the image height).
 * fwd = rnd(2^19 forward), right = rnd(2^18/f right), up = rnd(2^18/f up),
 * origin = rnd(2^16 (x, y, z)), rnd rounding half away from zero.
 * Errors: HF_E_INVALID_ARG (null out, w or h outside 1..HF_MAX_DIM,
 * hfov outside (0, 180)). */
int hf_camera_from_pose(double x, double y, double z, double yaw_deg, double pitch_deg,
                        double hfov_deg, uint32_t w, uint32_t h, hf_camera *out);

/* Host check of one camera against a W x H grid (the range limits above).
 * Returns HF_OK or HF_E_INVALID_ARG. */
int hf_validate_camera(uint32_t grid_w, uint32_t grid_h, const hf_camera *cam);

/* Host check of n cell words (the two-interval encoding above).
 * Returns HF_OK or HF_E_INVALID_ARG; *bad_index (may be NULL) gets the first bad word. */
int hf_validate_cells(const uint32_t *cells, size_t n, size_t *bad_index);

/* Host check of a width x height grid of paired texels (hf_pair_desc rules;
 * row_stride 0 = width).  Returns HF_OK or HF_E_INVALID_ARG; *bad_index (may
 * be NULL) gets y * width + x of the even texel of the first bad pair. */
int hf_validate_pairs(const uint16_t *texels, uint32_t width, uint32_t height, size_t row_stride,
                      size_t *bad_index);

/* Static text for one of the HF_E_* codes above (a library convention: the
 * paper defines no error reporting).  Never NULL; an unknown code gives
 * "unknown error". */
const char *hf_strerror(int code);

/* Sizes and device of a context.  Errors: HF_E_INVALID_ARG. */
int hf_info(const hf_ctx *ctx, hf_info_t *out);

/* Copy cells of a rectangle back to HOST memory as cell words (synchronous;
 * a paired-texel world is decoded).
 * Errors: HF_E_INVALID_ARG, HF_E_OUT_OF_BOUNDS, HF_E_CUDA. */
int hf_read_cells(hf_ctx *ctx, uint32_t x0, uint32_t y0, uint32_t w, uint32_t h,
                  uint32_t *out, size_t row_stride);

/* Copy pyramid level `level` (1..levels) to HOST memory (synchronous):
 * ceil(H/2^level) rows of ceil(W/2^level) node words, byte0 max h0, byte1 min
 * over cells of (slab ? h1 : 255), byte2 max over cells of (slab ? h2 : h0).
 * Errors: HF_E_INVALID_ARG, HF_E_CUDA. */
int hf_read_pyramid(hf_ctx *ctx, uint32_t level, uint32_t *out);

/* Rebuild the whole pyramid from the cells (the same kernels a full-grid edit
 * runs).  Errors: HF_E_INVALID_ARG, HF_E_CUDA. */
int hf_rebuild(hf_ctx *ctx);

/* Copy the per-cell shadow bounds last built by a render with HF_SHADOWS to
 * HOST memory (synchronous): W*H words, row-major, word = F | G << 16 with F
 * and G in units of 2^-8 world units: a shadow ray toward sun[] starting in
 * the cell (the cell it occupies just after t = 0) at height <= F*256 (in
 * 2^-16 units) is occluded, at height >= G*256 lit.  out may be NULL (only
 * sun[] is written); sun may be NULL.  The paper has no counterpart: its
 * shadow-map pass (Section 3) precomputes sun visibility approximately; these
 * bounds are exact but partial.
 * Errors: HF_E_INVALID_ARG (null ctx, or no bounds built), HF_E_CUDA. */
int hf_read_sun_bounds(hf_ctx *ctx, uint32_t *out, int32_t sun[3]);

/* Synchronise and read the fetch counters accumulated by HF_STATS renders:
 * out[0] pyramid node fetches, out[1] cell fetches, out[2] primary rays,
 * out[3] shadow rays, out[4] fetches made by shadow rays (a shadow-bound
 * lookup counts as one).  Clears them.
 * Errors: HF_E_INVALID_ARG, HF_E_CUDA. */
int hf_stats(hf_ctx *ctx, uint64_t out[5]);

/* ---------------------------------------------------------------- serving
 * A native serving loop over one resident world (the paper's interactive
 * setting: renders and edits interleaved, an edit visible to the next frame,
 * Section 4.4).  hf_serve_replay runs a stream of requests, each with its
 * arrival time, on the calling thread: a request becomes visible to the loop
 * when the host clock passes its arrival; renders are admitted in arrival
 * order into batches (up to max_batch requests, within output_budget bytes
 * of device output memory in flight) launched with hf_render on the first
 * free lane (one CUDA stream per lane, so batches overlap on the device);
 * an edit is applied with hf_edit when it reaches the head of the queue, so
 * renders admitted before it do not see it and every later one does; a batch
 * retires when its completion event has fired, and its output memory (from a
 * pool the loop owns, unless the request names its own buffers) is released.
 * Times are seconds from the start of the replay on the host clock:
 * `admitted` when the loop admitted the request (renders) or called hf_edit
 * (edits); `done` the device completion of the request's batch (renders) or
 * of the edit's copy and pyramid repair (edits).  Device times are mapped to
 * the host clock through a reference event whose host time is bracketed, before
 * the first request, by timed event round trips on an idle stream (the
 * bracket is a few microseconds wide).  The loop returns when every request
 * is done. */
#define HF_REQ_RENDER 0u
#define HF_REQ_EDIT 1u

typedef struct {
    uint32_t kind;        /* HF_REQ_RENDER or HF_REQ_EDIT */
    uint32_t reserved;    /* 0 */
    double arrival;       /* seconds after the start of the replay, non-decreasing */
    hf_camera cam;        /* HF_REQ_RENDER: the view */
    uint32_t x0, y0, w, h;/* HF_REQ_EDIT: the rectangle */
    const uint32_t *cells;/* HF_REQ_EDIT: w*h host cells, rows back to back (copied by hf_edit) */
    hf_outputs outs;      /* HF_REQ_RENDER, optional: caller-owned device buffers for the image
                             (a NULL member is not written); all NULL: the loop renders into its
                             own pool (counted against output_budget) and drops the image */
} hf_request;

typedef struct {
    double admitted;      /* host time of admission (renders) or of the hf_edit call (edits) */
    double done;          /* device completion of the batch (renders) or of the edit (edits) */
    uint32_t version;     /* edits applied before admission (renders); this edit's number (edits) */
    uint32_t batch;       /* batch index (renders); 0xFFFFFFFF for edits */
} hf_request_result;

typedef struct {
    uint32_t lanes;          /* CUDA streams with a batch in flight each, 1..64 */
    uint32_t max_batch;      /* renders per batch, 1..HF_MAX_CAMERAS */
    uint64_t output_budget;  /* bytes of device output memory in flight at once */
    uint32_t flags;          /* HF_SHADOWS (then a shadow byte per pixel is written too) */
    uint32_t tile_w, tile_h, mip_start;  /* as hf_render_opts (0 tile sides, HF_MIP_AUTO: defaults) */
} hf_serve_opts;

/* Runs reqs[0..n) and fills results[0..n).  HF_E_INVALID_ARG for a bad
 * option, a request of an unknown kind, arrivals out of order, or a render
 * whose outputs exceed the whole budget (nothing is run then); errors of
 * hf_render / hf_edit are returned as they occur (requests already launched
 * are completed first).  The lanes and the pool are created and destroyed
 * by the call. */
int hf_serve_replay(hf_ctx *ctx, const hf_request *reqs, uint32_t n, const hf_serve_opts *opts,
                    hf_request_result *results);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
