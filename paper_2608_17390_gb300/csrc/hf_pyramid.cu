// hf_pyramid.cu -- min/max pyramid build and incremental repair.
//
// Node (i, j) of level k covers cells [i 2^k, (i+1) 2^k) x [j 2^k, (j+1) 2^k)
// clipped to the grid; its word holds byte0 = max h0, byte1 = min over cells of
// (slab ? h1 : 255), byte2 = max over cells of (slab ? h2 : h0).  A node is
// the per-byte max/min of its (up to four) children, so after an edit of a cell
// rectangle only the nodes over that rectangle change, level by level: the
// "rebuild affected cells and their ancestors" of the paper's Sections 2 and
// 3.2, applied to a 2.5-D min/max hierarchy.  A full build is the repair of
// the whole grid, so build and repair run the same kernels.
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {
namespace {

constexpr uint32_t kIdentity = 0x0000FF00u;  // max h0 0, min h1 255, max top 0
constexpr int64_t kTailNodes = 4096;         // below this, finish in one block
constexpr int kTailThreads = 512;

__device__ __forceinline__ uint32_t cell_node(uint32_t c) {
    const uint32_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF, h2 = (c >> 16) & 0xFF;
    const bool slab = h1 > h0;
    return h0 | ((slab ? h1 : 255u) << 8) | ((slab ? h2 : h0) << 16);
}

// byte0 and byte2 by max, byte1 by min
__device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) {
    return (__vmaxu4(a, b) & 0x00FF00FFu) | (__vminu4(a, b) & 0x0000FF00u);
}

__device__ __forceinline__ uint32_t reduce_children(const uint32_t *src, uint32_t stride,
                                                    int32_t sw, int32_t sh, bool cells,
                                                    int32_t i, int32_t j) {
    uint32_t v = kIdentity;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int32_t x = 2 * i + dx, y = 2 * j + dy;
            if (x < sw && y < sh) {
                uint32_t c = src[(uint32_t)y * stride + (uint32_t)x];
                v = combine(v, cells ? cell_node(c) : c);
            }
        }
    }
    return v;
}

__global__ void k_pyr_level(const uint32_t *__restrict__ src, uint32_t src_stride, int32_t sw,
                            int32_t sh, int cells, uint32_t *__restrict__ dst,
                            uint32_t dst_stride, int32_t i0, int32_t j0, int32_t ni,
                            int64_t count) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count) return;
    const int32_t i = i0 + (int32_t)(idx % ni), j = j0 + (int32_t)(idx / ni);
    dst[(uint32_t)j * dst_stride + (uint32_t)i] =
        reduce_children(src, src_stride, sw, sh, cells != 0, i, j);
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
                reduce_children(src, w.stride[k - 1], sw, sh, k == 1, i, j);
        }
        __syncthreads();
    }
}

}  // namespace

int pyramid_repair(uint32_t *world, const WorldDev &w, int32_t x0, int32_t y0, int32_t x1,
                   int32_t y1, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (x1 <= x0 || y1 <= y0 || w.L == 0) return 0;
    int k = 1;
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
                                                         sh, k == 1, world + w.off[k],
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
