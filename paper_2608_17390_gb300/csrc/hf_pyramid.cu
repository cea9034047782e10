// hf_pyramid.cu -- min/max pyramid build and incremental repair.
//
// Node (i, j) of level k covers cells [i 2^k, (i+1) 2^k) x [j 2^k, (j+1) 2^k)
// clipped to the grid; its word holds byte0 = max h0, byte1 = min over cells of
// (slab ? h1 : 255), byte2 = max over cells of (slab ? h2 : h0).  A node is
// the per-byte max/min of its (up to four) children, so after an edit of a cell
// rectangle only the nodes over that rectangle change, level by level: the
// incremental repair of the paper's Sections 2 and 3.2 (the edited cells, then
// the nodes above them), applied to a 2.5-D min/max hierarchy.  The full build (hf_create,
// hf_rebuild) makes levels 1..6 per 64 x 64 tile in shared memory so the cells
// are read from HBM once; repair recomputes the nodes over a rectangle level by
// level.  The two paths share only the byte-wise combine, and the tests compare
// each with the oracle's pyramid.
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {
namespace {

constexpr uint32_t kIdentity = 0x0000FF00u;  // max h0 0, min h1 255, max top 0
constexpr int64_t kTailNodes = 4096;         // below this, finish in one block
constexpr int kTailThreads = 512;

// Level-0 words are stored in node form (cell_encode); the node of one cell
// is its word without the material byte.
__device__ __forceinline__ uint32_t cell_node(uint32_t c) { return c & 0x00FFFFFFu; }

__global__ void k_cells_encode(uint32_t *__restrict__ cells, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cells[i] = cell_encode(cells[i]);
}

// byte0 and byte2 by max, byte1 by min (each field compared in place)
__device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) {
    return max(a & 0x0000FFu, b & 0x0000FFu) | min(a & 0x00FF00u, b & 0x00FF00u) |
           max(a & 0xFF0000u, b & 0xFF0000u);
}

// Child (x, y) of a level-1 node or of a higher one.  src_mode: 0 node words,
// 1 level-0 cells in node form, 2 level-0 paired texels (rows of stride / 2
// words, stride = width in cells).
__device__ __forceinline__ uint32_t child_node(const uint32_t *src, uint32_t stride, int src_mode,
                                               int32_t x, int32_t y) {
    if (src_mode == 2)
        return cell_node(pair_node(src[(uint32_t)y * (stride >> 1) + ((uint32_t)x >> 1)],
                                   (uint32_t)x & 1));
    const uint32_t c = src[(uint32_t)y * stride + (uint32_t)x];
    return src_mode ? cell_node(c) : c;
}

__device__ __forceinline__ uint32_t reduce_children(const uint32_t *src, uint32_t stride,
                                                    int32_t sw, int32_t sh, int src_mode,
                                                    int32_t i, int32_t j) {
    uint32_t v = kIdentity;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int32_t x = 2 * i + dx, y = 2 * j + dy;
            if (x < sw && y < sh) v = combine(v, child_node(src, stride, src_mode, x, y));
        }
    }
    return v;
}

__global__ void k_pyr_level(const uint32_t *__restrict__ src, uint32_t src_stride, int32_t sw,
                            int32_t sh, int src_mode, uint32_t *__restrict__ dst,
                            uint32_t dst_stride, int32_t i0, int32_t j0, int32_t ni,
                            int64_t count) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count) return;
    const int32_t i = i0 + (int32_t)(idx % ni), j = j0 + (int32_t)(idx / ni);
    dst[(uint32_t)j * dst_stride + (uint32_t)i] =
        reduce_children(src, src_stride, sw, sh, src_mode, i, j);
}

// Levels k_from..L of a small rectangle in one block; __syncthreads orders
// the levels (the block's own global writes are visible to it after a barrier).
__global__ void __launch_bounds__(kTailThreads) k_pyr_tail(uint32_t *world, const WorldDev w,
                                                           int32_t k_from, int32_t x0,
                                                           int32_t y0, int32_t x1, int32_t y1) {
    for (int k = k_from; k <= w.L; ++k) {
        const int32_t i0 = x0 >> k, i1 = (x1 - 1) >> k, j0 = y0 >> k, j1 = (y1 - 1) >> k;
        const int32_t ni = i1 - i0 + 1, nj = j1 - j0 + 1;
        const int32_t sw = k == 1 ? w.W : (w.W + (1 << (k - 1)) - 1) >> (k - 1);
        const int32_t sh = k == 1 ? w.H : (w.H + (1 << (k - 1)) - 1) >> (k - 1);
        const uint32_t *src = world + w.off[k - 1];
        uint32_t *dst = world + w.off[k];
        for (int32_t idx = threadIdx.x; idx < ni * nj; idx += blockDim.x) {
            const int32_t i = i0 + idx % ni, j = j0 + idx / ni;
            dst[(uint32_t)j * w.stride[k] + (uint32_t)i] =
                reduce_children(src, w.stride[k - 1], sw, sh, k == 1 ? 1 + w.pair : 0, i, j);
        }
        __syncthreads();
    }
}

// Full build, levels 1..min(6, L) of one 64 x 64 cell tile per block: the
// cells are read from HBM once (coalesced), every level of the tile is made in
// shared memory from the one below, and each level is written once.
constexpr int kTile = 64;
constexpr int kTileLevels = 6;  // 64 -> 1
constexpr int kBuildThreads = 256;

__global__ void __launch_bounds__(kBuildThreads) k_pyr_build_tiles(uint32_t *world,
                                                                   const WorldDev w,
                                                                   int32_t top) {
    // level-2 nodes of the tile (16 x 16), then levels 3..6 back to back
    __shared__ uint32_t s_lv[16 * 16 + 8 * 8 + 4 * 4 + 2 * 2 + 1];
    const int32_t bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
    // this thread's 4 x 4 cell block inside the tile
    const int qx = threadIdx.x & 15, qy = threadIdx.x >> 4;
    const int32_t cx0 = bx + 4 * qx, cy0 = by + 4 * qy;
    const uint32_t *cells = world;  // level 0
    uint32_t c[4][4];
    if (cx0 + 4 <= w.W && cy0 + 4 <= w.H && (w.W & 3) == 0 && !w.pair) {
        uint4 v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)  // four 16-byte loads issued before use
            v[r] = __ldg(reinterpret_cast<const uint4 *>(cells + (uint32_t)(cy0 + r) * (uint32_t)w.W +
                                                         (uint32_t)cx0));
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            c[r][0] = cell_node(v[r].x);
            c[r][1] = cell_node(v[r].y);
            c[r][2] = cell_node(v[r].z);
            c[r][3] = cell_node(v[r].w);
        }
    } else if (cx0 + 4 <= w.W && cy0 + 4 <= w.H && (w.W & 3) == 0) {
        // paired texels: the 4 cells of a row are 2 pair words (8 bytes,
        // aligned because W / 2 and cx0 / 2 are even)
        uint2 v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            v[r] = __ldg(reinterpret_cast<const uint2 *>(
                cells + (uint32_t)(cy0 + r) * ((uint32_t)w.W >> 1) + ((uint32_t)cx0 >> 1)));
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            c[r][0] = cell_node(pair_node(v[r].x, 0));
            c[r][1] = cell_node(pair_node(v[r].x, 1));
            c[r][2] = cell_node(pair_node(v[r].y, 0));
            c[r][3] = cell_node(pair_node(v[r].y, 1));
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t x = cx0 + q, y = cy0 + r;
                c[r][q] = (x < w.W && y < w.H) ? child_node(cells, (uint32_t)w.W, 1 + w.pair, x, y)
                                               : kIdentity;
            }
    }
    // levels 1 and 2 of the block in registers
    uint32_t l1[2][2];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
            l1[b][a] = combine(combine(c[2 * b][2 * a], c[2 * b][2 * a + 1]),
                               combine(c[2 * b + 1][2 * a], c[2 * b + 1][2 * a + 1]));
    const uint32_t l2 = combine(combine(l1[0][0], l1[0][1]), combine(l1[1][0], l1[1][1]));
    {
        const int32_t gx = cx0 >> 1, gy = cy0 >> 1;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                if ((uint32_t)(gx + a) < w.stride[1] && (uint32_t)(gy + b) < w.rows[1])
                    world[w.off[1] + (uint32_t)(gy + b) * w.stride[1] + (uint32_t)(gx + a)] =
                        l1[b][a];
    }
    if (top >= 2) {
        const int32_t gx = cx0 >> 2, gy = cy0 >> 2;
        if ((uint32_t)gx < w.stride[2] && (uint32_t)gy < w.rows[2])
            world[w.off[2] + (uint32_t)gy * w.stride[2] + (uint32_t)gx] = l2;
    }
    s_lv[threadIdx.x] = l2;
    __syncthreads();
    // levels 3..top from the 16 x 16 level-2 nodes in shared memory
    int n = 16, src = 0, dst = 256;
    for (int k = 3; k <= top; ++k) {
        const int m = n >> 1;
        const int32_t ox = bx >> k, oy = by >> k;  // tile origin at level k
        if (threadIdx.x < m * m) {
            const int a = threadIdx.x % m, b = threadIdx.x / m;
            const uint32_t *p0 = s_lv + src + (2 * b) * n + 2 * a;
            const uint32_t v = combine(combine(p0[0], p0[1]), combine(p0[n], p0[n + 1]));
            s_lv[dst + threadIdx.x] = v;
            const int32_t gx = ox + a, gy = oy + b;
            if ((uint32_t)gx < w.stride[k] && (uint32_t)gy < w.rows[k])
                world[w.off[k] + (uint32_t)gy * w.stride[k] + (uint32_t)gx] = v;
        }
        __syncthreads();
        src = dst;
        dst += m * m;
        n = m;
    }
}

}  // namespace

int cells_encode(uint32_t *cells, uint32_t n, void *stream) {
    if (n == 0) return 0;
    const uint32_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_cells_encode<<<blocks, 256, 0, (cudaStream_t)stream>>>(cells, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pyramid_build(uint32_t *world, const WorldDev &w, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (w.L == 0) return 0;
    const int top = w.L < kTileLevels ? w.L : kTileLevels;
    const dim3 grid((w.W + kTile - 1) / kTile, (w.H + kTile - 1) / kTile);
    k_pyr_build_tiles<<<grid, kBuildThreads, 0, s>>>(world, w, top);
    if (cudaGetLastError() != cudaSuccess) return -1;
    if (top == w.L) return 0;
    // levels top+1 .. L from level `top`, over the whole grid (small)
    return pyramid_repair_from(world, w, top + 1, 0, 0, w.W, w.H, stream);
}

int pyramid_repair(uint32_t *world, const WorldDev &w, int32_t x0, int32_t y0, int32_t x1,
                   int32_t y1, void *stream) {
    return pyramid_repair_from(world, w, 1, x0, y0, x1, y1, stream);
}

int pyramid_repair_from(uint32_t *world, const WorldDev &w, int k_from, int32_t x0, int32_t y0,
                        int32_t x1, int32_t y1, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (x1 <= x0 || y1 <= y0 || w.L == 0 || k_from > w.L) return 0;
    int k = k_from;
    for (; k <= w.L; ++k) {
        const int32_t i0 = x0 >> k, i1 = (x1 - 1) >> k, j0 = y0 >> k, j1 = (y1 - 1) >> k;
        const int64_t ni = i1 - i0 + 1, nj = j1 - j0 + 1;
        const int64_t count = ni * nj;
        if (count <= kTailNodes) break;
        const int32_t sw = (w.W + (1 << (k - 1)) - 1) >> (k - 1);
        const int32_t sh = (w.H + (1 << (k - 1)) - 1) >> (k - 1);
        const int threads = 256;
        const int64_t blocks = (count + threads - 1) / threads;
        k_pyr_level<<<(unsigned)blocks, threads, 0, s>>>(world + w.off[k - 1], w.stride[k - 1], sw,
                                                         sh, k == 1 ? 1 + w.pair : 0,
                                                         world + w.off[k],
                                                         w.stride[k], i0, j0, (int32_t)ni, count);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    if (k <= w.L) {
        k_pyr_tail<<<1, kTailThreads, 0, s>>>(world, w, k, x0, y0, x1, y1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

}  // namespace hf
