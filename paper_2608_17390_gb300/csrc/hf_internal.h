// hf_internal.h -- device-side structures shared by the kernels and the C ABI.
//
// Memory layout in HBM (one allocation per context, 256-byte aligned levels):
//   level 0   : the cells, W x H uint32 words, row-major y*W + x, each in node
//               form with its material (cell_encode below); or, for a world
//               created from paired texels, W x H uint16 texels (pair_node)
//   level k>=1: ceil(W/2^k) x ceil(H/2^k) node words, row-major,
//               byte0 max h0, byte1 min (slab ? h1 : 255), byte2 max (slab ? h2 : h0)
// Per-render scratch (one block per render slot):
//   BatchHeader (tile counter, camera count, tile count), then CamDev[n].
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

struct hf_ctx;  // the C ABI's opaque context (hf_api.cpp)

namespace hf {

// A valid cell word (byte0 h0, byte1 h1, byte2 h2, byte3 material; a slab
// when h1 > h0, else h1 = h2 = 0) in the node form of a one-cell pyramid
// node: byte0 h0, byte1 (slab ? h1 : 255), byte2 (slab ? h2 : h0), material
// kept in byte3.  Slab cells are unchanged; the map is one to one on valid
// cells (a slab exactly when byte2 > byte0), so level 0 is stored this way
// and every traversal level reads the same word layout.
__host__ __device__ inline uint32_t cell_encode(uint32_t c) {
    const uint32_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF;
    return h1 > h0 ? c : (c & 0xFF0000FFu) | 0xFF00u | (h0 << 16);
}
// Inverse of cell_encode.
__host__ __device__ inline uint32_t cell_decode(uint32_t n) {
    const uint32_t b0 = n & 0xFF, b2 = (n >> 16) & 0xFF;
    return b2 > b0 ? n : (n & 0xFF0000FFu);
}

// The node-form word (with material) of cell `odd` (0 even, 1 odd) of a pair
// of 2-byte texels loaded as one little-endian 32-bit word: altitude and meta
// byte of the even texel, then of the odd one.  Meta bit 7: the pair is
// double-level; bits 6..3: a delta nibble; bits 2..0: material.  A
// double-level pair is one column for both cells, floor top = even altitude,
// slab top = odd altitude, slab underside = slab top - (16 * even nibble +
// odd nibble) (the data section's pair encoding, with this bit layout).
__host__ __device__ inline uint32_t pair_node(uint32_t pw, uint32_t odd) {
    const uint32_t ve = pw & 0xFF, me = (pw >> 8) & 0xFF, vo = (pw >> 16) & 0xFF, mo = pw >> 24;
    const uint32_t mat = (odd ? mo : me) & 7;
    if (me & 0x80) {
        const uint32_t mid = vo - (((me << 1) & 0xF0) | ((mo >> 3) & 0x0F));
        return ve | (mid << 8) | (vo << 16) | (mat << 24);
    }
    const uint32_t v = odd ? vo : ve;
    return v | 0xFF00u | (v << 16) | (mat << 24);
}

// Shading (this library's fixed choice; the paper names its terms only): an
// 8-entry albedo table by material, ambient 0.3, diffuse 0.7, a sky colour.
#define HF_ALBEDO_TABLE                                                                     \
    {{0.55f, 0.50f, 0.40f}, {0.35f, 0.55f, 0.25f}, {0.60f, 0.60f, 0.62f}, {0.80f, 0.72f, 0.50f}, \
     {0.30f, 0.30f, 0.32f}, {0.70f, 0.35f, 0.20f}, {0.90f, 0.90f, 0.95f}, {0.25f, 0.40f, 0.60f}}
constexpr float kAmbient = 0.3f, kDiffuse = 0.7f;
constexpr uint32_t kSkyColour = 0xFFEBB487u;  // r 135, g 180, b 235, a 255

constexpr int kMaxLevels = 14;  // 2^14 = 16384 = largest grid side
constexpr int kShift = 16;      // 2^16 fixed-point units per world unit
#ifndef HF_TRACE_THREADS
#define HF_TRACE_THREADS 256  // measured: 128 / 256 / 512 (256: 0.4 % faster than 128)
#endif
constexpr int kThreads = HF_TRACE_THREADS;  // threads per trace block (8 warps)
constexpr uint32_t kMaxCams = 4096;
constexpr uint32_t kDefaultMipStart = 6;  // coarsest level used when the caller asks for the default
#ifndef HF_SHADOW_MIP_EXTRA
#define HF_SHADOW_MIP_EXTRA 4
#endif
// shadow rays may climb this many levels higher than primary rays
constexpr uint32_t kShadowMipExtra = HF_SHADOW_MIP_EXTRA;
#ifndef HF_SHADOW_START
#define HF_SHADOW_START 0
#endif
// level at which a shadow ray starts: its origin lies next to a surface, so
// the coarse nodes around it are rarely empty; it climbs as it leaves them
constexpr int kShadowStart = HF_SHADOW_START;

constexpr uint8_t kFaceNX = 0, kFacePX = 1, kFaceNY = 2, kFacePY = 3, kFaceNZ = 4, kFacePZ = 5,
                  kFaceInside = 6, kFaceError = 254, kFaceMiss = 255;

struct WorldDev {
    const uint32_t *base;               // level 0 at base, level k at base + off[k]
    uint32_t off[kMaxLevels + 1];       // word offset of each level
    uint32_t stride[kMaxLevels + 1];    // width of each level in nodes (cells at level 0) = its
                                        // words per row, except for paired texels (W / 2)
    uint32_t rows[kMaxLevels + 1];      // rows of each level (= its height in nodes)
    int32_t W, H, L;                    // grid size, top level
    int32_t pair;                       // 1: level 0 holds paired 2-byte texels
};

#ifdef __CUDACC__
// Node-form word of cell (x, y) of level 0, either storage.
__device__ __forceinline__ uint32_t level0_node(const WorldDev &w, int32_t x, int32_t y) {
    if (w.pair)
        return pair_node(__ldg(w.base + (uint32_t)y * ((uint32_t)w.W >> 1) + ((uint32_t)x >> 1)),
                         (uint32_t)x & 1);
    return __ldg(w.base + (uint32_t)y * (uint32_t)w.W + (uint32_t)x);
}
#endif

struct CamDev {
    int32_t o[3];
    int32_t F[3], R[3], U[3];
    uint32_t w, h;
    uint32_t tiles_x, tile_base;  // tiles per image row, first global tile of this camera
    uint32_t *hit_cell;
    uint8_t *layer;
    uint8_t *face;
    float *depth;
    uint32_t *rgba;
    uint8_t *shadow;
};

struct BatchHeader {
    uint32_t counter;      // next global tile (atomic, zero at launch)
    uint32_t n_cams;
    uint32_t total_tiles;
    uint32_t pad[29];      // CamDev array starts 128 bytes in
};
static_assert(sizeof(BatchHeader) == 128, "header size");

struct RenderParams {
    WorldDev world;
    BatchHeader *hdr;              // per-slot scratch header (batched kernel)
    const CamDev *cams;            // per-slot camera table
    uint32_t *status;              // bit 0: a ray hit its step guard
    unsigned long long *stats;     // 5 counters (HF_STATS)
    int32_t tile_w_log2, tile_h_log2;
    int32_t mip_start;             // coarsest level for primary rays
    int32_t shadow_mip;            // coarsest level for shadow rays
    int32_t max_steps;
    int32_t sun[3];
    float sun_n[3];                // sun / |sun|
    const uint32_t *sun_bounds;    // per-cell shadow bounds for `sun` (hf_sun.cu), or null
    const uint32_t *prefetch;      // start of the world levels the trace kernels warm in L2
    uint32_t prefetch_lines;       // 128-byte lines from `prefetch` (0: none)
};

// Parameters of the fixed-step comparison marcher (hf_march.cu).
struct MarchParams {
    int32_t steps;       // forward samples over the clipped segment
    int32_t bisections;  // halvings of the bracketing interval
    float far_dist;      // world units
};
int launch_march_batched(const RenderParams &p, const MarchParams &m, int blocks, void *stream);
int march_occupancy(int *blocks_per_sm);

// Parameters of the scattered comparison renderer (hf_scatter.cu).  The
// per-camera footprints (float4: s_lo, s_hi, k_lat, u_min) follow the camera
// table in the slot scratch.
struct ScatterParams {
    uint32_t nu, nv, nz;     // footprint samples across and along; points per column interval
    uint32_t max_pixels;     // largest w * h of the batch
    float depth_max;         // depth quantisation range (world units)
    uint32_t colour[8];      // resolved colour per material (an up-facing, lit surface)
    int32_t raw;             // 1: leave the packed words in hit_cell, no resolve
};
int launch_scatter(const RenderParams &p, const ScatterParams &s, uint32_t n_cams, void *stream);

// The voxel occupancy pyramid of the RayVoxel comparison renderer
// (hf_voxel.cu): level l of nx x ny x nz voxels in Morton-coded 8^3 tiles of
// tx x ty x tz tiles, 16 words each, starting at word off[l].
constexpr int kVoxMaxLevels = 16;
constexpr int kVoxMaxLayers = 256;  // nz0 = ceil(256 / vz), vz >= 1
struct VoxelDev {
    uint32_t *words;
    uint32_t off[kVoxMaxLevels];
    int32_t nx[kVoxMaxLevels], ny[kVoxMaxLevels], nz[kVoxMaxLevels];
    int32_t tx[kVoxMaxLevels], ty[kVoxMaxLevels];
    int32_t vx, vy, vz, levels;
};
struct VoxelParams {
    int32_t outer;    // traversal steps allowed per ray
    int32_t inner;    // samples per occupied leaf voxel
    float far_dist;   // world units
};
// Recompute the voxels over cell rectangle [x0, x1) x [y0, y1), every level
// (fresh: the words are zero, as after allocation).
int voxel_repair(const WorldDev &w, const VoxelDev &v, int32_t x0, int32_t y0, int32_t x1,
                 int32_t y1, bool fresh, void *stream);
int launch_voxel_trace(const RenderParams &p, const VoxelDev &v, const VoxelParams &q,
                       uint32_t n_cams, uint32_t max_pixels, void *stream);

// Launch wrappers (hf_trace.cu)
// The trace kernels are instantiated per level-0 storage; p.world.pair picks one.
int launch_trace_batched(const RenderParams &p, bool shadows, bool stats, int blocks,
                         void *stream);
// (the plain kernel takes its camera record as a launch parameter)
int launch_trace_plain(const RenderParams &p, bool shadows, bool stats, const CamDev &cam,
                       uint32_t n_tiles, void *stream);
const void *trace_batched_fn(bool shadows, bool stats, bool pair);
int trace_batched_occupancy(bool shadows, bool stats, bool pair, int *blocks_per_sm);

// What the allocation-free render needs to know about a context (hf_api.cpp).
struct CtxView {
    WorldDev world;
    void *stream;
    int device;
    int sm_count;
    int occ_shadows[2];  // batched-kernel blocks per SM without / with shadow rays
};
int ctx_view(const ::hf_ctx *ctx, CtxView *out);

// Shadow bounds (hf_sun.cu): per cell, F | G << 16 in 2^-8 world units: a
// shadow ray toward `sun` starting in the cell at height <= F << 8 is
// occluded, at >= G << 8 lit.  Only for rising, non-vertical suns whose rays
// clear the 255-unit height range within kSunMaxReach cells.
constexpr int64_t kSunMaxReach = 1024;
bool sun_bounds_eligible(const int32_t sun[3]);
// Bytes of the bounds buffer of a W x H grid: the W * H words, then a table
// of the sun's row offsets per column of travel that the build fills and the
// repair reads.
size_t sun_bounds_bytes(int32_t W, int32_t H);
// Recompute the bounds of the cells of [x0, x1) x [y0, y1) from the cells.
int sun_bounds(const WorldDev &w, uint32_t *bounds, const int32_t sun[3], int32_t x0, int32_t y0,
               int32_t x1, int32_t y1, void *stream);
// Recompute, after an edit of the cells of [x0, x1) x [y0, y1), the bounds
// that depend on them (the pyramid must already be repaired).
int sun_bounds_repair(const WorldDev &w, uint32_t *bounds, const int32_t sun[3], int32_t x0,
                      int32_t y0, int32_t x1, int32_t y1, void *stream);
// The cells whose bounds depend on the cells of [x0, x1) x [y0, y1) lie in
// out = {x0', y0', x1', y1'} (clipped to the grid).
void sun_bounds_region(const WorldDev &w, const int32_t sun[3], int32_t x0, int32_t y0,
                       int32_t x1, int32_t y1, int32_t *out);

// Pyramid (hf_pyramid.cu): repair the nodes covering cell rectangle
// [x0, x1) x [y0, y1) at every level 1..L, in order.
int pyramid_repair(uint32_t *world, const WorldDev &w, int32_t x0, int32_t y0, int32_t x1,
                   int32_t y1, void *stream);
// Same, for levels k_from..L only (levels below k_from must already be current).
int pyramid_repair_from(uint32_t *world, const WorldDev &w, int k_from, int32_t x0, int32_t y0,
                        int32_t x1, int32_t y1, void *stream);
// Encode the W x H cells just copied to level 0 into node form, in place.
int cells_encode(uint32_t *cells, uint32_t n, void *stream);
// Full build of levels 1..L from the cells: levels 1..6 by 64 x 64 tiles in
// shared memory (cells read once), the rest by repair of the whole grid.
int pyramid_build(uint32_t *world, const WorldDev &w, void *stream);

}  // namespace hf
