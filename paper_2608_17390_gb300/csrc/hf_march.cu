// hf_march.cu -- the paper's fixed-step height-field ray march (its Section
// 3.1), as a comparison kernel for the exact cast.
//
// Per pixel ray p(t) = o + t d in world units (o = origin / 2^16, d = integer
// direction / 2^16, the same parameter t as the exact cast): the segment is
// clipped at the far distance and, for a descending ray, at z = 0; `steps`
// samples are spaced uniformly over it; the first sample whose point is solid
// (z <= low, or mid <= z <= high, of the cell containing it) stops the search
// and `bisections` halvings keep the solid end.  A ray with no solid sample
// misses.  All arithmetic is float32, round to nearest, with no fused
// multiply-add, in a fixed order, so results are reproducible bit for bit.
// The method can step over features thinner than its sample spacing (the
// trade-off the paper states); the exact cast cannot.
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {
namespace {

struct MarchPoint {
    bool solid;
    int32_t cx, cy;
    uint8_t layer;
};

__device__ __forceinline__ MarchPoint march_solid(const WorldDev &w, float x, float y, float z) {
    MarchPoint r;
    r.cx = (int32_t)floorf(x);
    r.cy = (int32_t)floorf(y);
    r.solid = false;
    r.layer = 0;
    if ((uint32_t)r.cx < (uint32_t)w.W && (uint32_t)r.cy < (uint32_t)w.H) {
        const uint32_t c = level0_node(w, r.cx, r.cy);
        const uint32_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF, h2 = (c >> 16) & 0xFF;
        const bool floor_ = z <= (float)h0;
        const bool upper = h2 > h0 && z >= (float)h1 && z <= (float)h2;  // node-form cell
        r.solid = floor_ || upper;
        r.layer = floor_ ? 0 : 1;
    }
    return r;
}

__device__ __forceinline__ void march_pixel(const RenderParams &p, const MarchParams &m,
                                            const CamDev &c, int32_t px, int32_t py) {
    const int32_t a = 2 * px + 1 - (int32_t)c.w;
    const int32_t b = (int32_t)c.h - 1 - 2 * py;
    const float inv_s = 1.0f / 65536.0f;
    const float ox = __fmul_rn(__int2float_rn(c.o[0]), inv_s);
    const float oy = __fmul_rn(__int2float_rn(c.o[1]), inv_s);
    const float oz = __fmul_rn(__int2float_rn(c.o[2]), inv_s);
    const float dx = __fmul_rn(__int2float_rn(c.F[0] + a * c.R[0] + b * c.U[0]), inv_s);
    const float dy = __fmul_rn(__int2float_rn(c.F[1] + a * c.R[1] + b * c.U[1]), inv_s);
    const float dz = __fmul_rn(__int2float_rn(c.F[2] + a * c.R[2] + b * c.U[2]), inv_s);
    float sq = __fmul_rn(dx, dx);
    sq = __fadd_rn(sq, __fmul_rn(dy, dy));
    sq = __fadd_rn(sq, __fmul_rn(dz, dz));
    const float len = __fsqrt_rn(sq);
    float t_end = __fdiv_rn(m.far_dist, len);
    if (dz < 0.0f) {
        const float tz = __fdiv_rn(-oz, dz);
        if (tz < t_end) t_end = tz;
    }
    const float dt = __fdiv_rn(t_end, (float)(m.steps + 1));
    bool found = false;
    float ta = 0.0f, tb = 0.0f;
    for (int i = 1; i <= m.steps; ++i) {
        const float t = __fmul_rn((float)i, dt);
        const MarchPoint q = march_solid(p.world, __fadd_rn(ox, __fmul_rn(t, dx)),
                                         __fadd_rn(oy, __fmul_rn(t, dy)),
                                         __fadd_rn(oz, __fmul_rn(t, dz)));
        if (q.solid) {
            found = true;
            tb = t;
            ta = __fmul_rn((float)(i - 1), dt);
            break;
        }
    }
    uint32_t cell = 0xFFFFFFFFu;
    uint8_t layer = 255;
    float depth = __int_as_float(0x7f800000);
    if (found) {
        for (int k = 0; k < m.bisections; ++k) {
            const float tm = __fmul_rn(__fadd_rn(ta, tb), 0.5f);
            const MarchPoint q = march_solid(p.world, __fadd_rn(ox, __fmul_rn(tm, dx)),
                                             __fadd_rn(oy, __fmul_rn(tm, dy)),
                                             __fadd_rn(oz, __fmul_rn(tm, dz)));
            if (q.solid) tb = tm;
            else ta = tm;
        }
        const MarchPoint q = march_solid(p.world, __fadd_rn(ox, __fmul_rn(tb, dx)),
                                         __fadd_rn(oy, __fmul_rn(tb, dy)),
                                         __fadd_rn(oz, __fmul_rn(tb, dz)));
        cell = (uint32_t)q.cy * (uint32_t)p.world.W + (uint32_t)q.cx;
        layer = q.layer;
        depth = __fmul_rn(tb, len);
    }
    const uint32_t pix = (uint32_t)py * c.w + (uint32_t)px;
    if (c.hit_cell) __stcs(c.hit_cell + pix, cell);
    if (c.layer) __stcs(c.layer + pix, layer);
    if (c.depth) __stcs(c.depth + pix, depth);
}

__device__ __forceinline__ const CamDev &stage(CamDev *slot, const CamDev *cams, uint32_t i,
                                               int lane) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(cams + i);
    uint32_t *dst = reinterpret_cast<uint32_t *>(slot);
    __syncwarp();
    if (lane < (int)(sizeof(CamDev) / 4)) dst[lane] = src[lane];
    __syncwarp();
    return *slot;
}

// Persistent: warps pop (camera, tile) items from the batch's atomic counter.
__global__ void __launch_bounds__(kThreads) k_march_batched(const RenderParams p,
                                                            const MarchParams m) {
    __shared__ uint32_t s_base[kMaxCams + 1];
    __shared__ CamDev s_cam[kThreads / 32];
    const uint32_t n = p.hdr->n_cams;
    const uint32_t total = p.hdr->total_tiles;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s_base[i] = p.cams[i].tile_base;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&p.hdr->counter, 1u);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (t >= total) break;
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_base[mid] <= t) lo = mid;
            else hi = mid;
        }
        const CamDev &c = stage(&s_cam[threadIdx.x >> 5], p.cams, lo, lane);
        const uint32_t local = t - s_base[lo];
        const uint32_t tx = local % c.tiles_x, ty = local / c.tiles_x;
        const int32_t x0 = (int32_t)tx << p.tile_w_log2, y0 = (int32_t)ty << p.tile_h_log2;
        const int32_t npix = 1 << (p.tile_w_log2 + p.tile_h_log2);
        for (int i = lane; i < npix; i += 32) {
            const int32_t px = x0 + (i & ((1 << p.tile_w_log2) - 1));
            const int32_t py = y0 + (i >> p.tile_w_log2);
            if (px < (int32_t)c.w && py < (int32_t)c.h) march_pixel(p, m, c, px, py);
        }
    }
}

}  // namespace

int launch_march_batched(const RenderParams &p, const MarchParams &m, int blocks, void *stream) {
    k_march_batched<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(p, m);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int march_occupancy(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               blocks_per_sm, reinterpret_cast<const void *>(&k_march_batched), kThreads, 0) ==
                   cudaSuccess
               ? 0
               : -1;
}

}  // namespace hf
