// hf_voxel.cu -- the paper's voxel-accelerated ray march, RayVoxel (its
// Section 3), as a comparison renderer: a conservative occupancy pyramid and a
// hierarchical DDA with fixed sampling at the leaves.
//
// Occupancy.  Level-0 voxel (i, j, k) covers cells [i vx, (i+1) vx) x
// [j vy, (j+1) vy) and heights [k vz, (k+1) vz] (closed); it is occupied when
// some cell there is solid at some such height (z0 <= h0, or a slab with
// h1 <= z1 and z0 <= h2).  Level l+1 voxel = OR of its eight level-l children.
// Each level is stored as Morton-coded 8 x 8 x 8 tiles of bits: tile
// (tx, ty, tz) at (tz TY + ty) TX + tx, 16 words of 32 bits each, voxel bit
// morton3(x & 7, y & 7, z & 7) (bits of x, y, z interleaved from the lowest).
//
// Traversal (one thread per pixel; float32, round to nearest, no fused
// multiply-add, in a fixed order, so results are reproducible bit for bit):
// clip the ray to the voxel grid's box and the far distance; start at the top
// level; an empty voxel advances to its exit plane (climbing a level when the
// crossed plane is a parent boundary); an occupied one is opened (the child
// the ray is in just after t: the first child along the direction on the axis
// last crossed, else the one holding p(t)); an occupied leaf is sampled at
// `inner` midpoints of the ray's stretch inside it, and the first SOLID sample
// is the hit.  Thin features can slip between samples (the paper's trade-off).
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hf {
namespace {

constexpr int kVoxThreads = 128;

__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// word index and bit of voxel (x, y, z) of level l
__device__ __forceinline__ void vox_addr(const VoxelDev &v, int l, uint32_t x, uint32_t y,
                                         uint32_t z, uint32_t &word, uint32_t &bit) {
    const uint32_t tile = ((z >> 3) * v.ty[l] + (y >> 3)) * v.tx[l] + (x >> 3);
    const uint32_t m = morton3(x & 7, y & 7, z & 7);
    word = v.off[l] + tile * 16 + (m >> 5);
    bit = m & 31;
}

// One level of the pyramid as the traversal reads it: a per-block shared
// table, so lanes at different levels read it in one shared-memory access
// (kernel parameters indexed by a per-lane level would serialise).
struct __align__(16) VoxLevel {
    uint32_t off;
    int32_t tx, ty, pad0;
    int32_t n[3], pad1;
};

__device__ __forceinline__ bool vox_occupied(const VoxelDev &v, const VoxLevel &lv, uint32_t x,
                                             uint32_t y, uint32_t z) {
    const uint32_t tile = ((z >> 3) * (uint32_t)lv.ty + (y >> 3)) * (uint32_t)lv.tx + (x >> 3);
    const uint32_t m = morton3(x & 7, y & 7, z & 7);
    return (__ldg(v.words + lv.off + tile * 16 + (m >> 5)) >> (m & 31)) & 1u;
}

// leaf sample fractions (s + 0.5) / inner held in shared memory up to this count
constexpr int kVoxFracTable = 64;

// log2 of a power-of-two voxel extent, else -1
__host__ __device__ __forceinline__ int32_t pow2_log2(int32_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int32_t e = 0;
    while ((1 << e) < v) ++e;
    return e;
}

// The correctly rounded quotient pk / (vs 2^l).  For a power-of-two extent
// (vs = 2^e) it is the correctly rounded product pk 2^-(e+l): both round the
// same real number, and 2^-(e+l) (at least 2^-21) is an exact float.
__device__ __forceinline__ float vox_quot(float pk, int32_t vs, int32_t vs_log2, int l) {
    if (vs_log2 >= 0) return __fmul_rn(pk, __int_as_float((127 - vs_log2 - l) << 23));
    return __fdiv_rn(pk, (float)(vs << l));
}

__device__ __forceinline__ bool vox_occupied(const VoxelDev &v, int l, uint32_t x, uint32_t y,
                                             uint32_t z) {
    uint32_t w, b;
    vox_addr(v, l, x, y, z, w, b);
    return (__ldg(v.words + w) >> b) & 1u;
}


// Level-0 voxel columns [i0, i0+ni) x [j0, j0+nj): the layers each column's
// cells occupy, gathered as a bit mask, then written into the column's bits.
// In an 8^3 tile the layers 2q and 2q+1 of one column share a word (the bits
// morton and morton + 4), so one atomic pair per word updates them; a fresh
// build (zeroed words) needs only the OR.
__global__ void k_vox_level0(const WorldDev w, const VoxelDev v, int32_t i0, int32_t j0,
                             int32_t ni, int32_t nj, int fresh) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * nj) return;
    const int32_t i = i0 + t % ni, j = j0 + t / ni;
    uint32_t mask[kVoxMaxLayers / 32];
#pragma unroll
    for (int q = 0; q < kVoxMaxLayers / 32; ++q) mask[q] = 0;
    const int32_t nz = v.nz[0];
    for (int32_t y = j * v.vy; y < min((j + 1) * v.vy, w.H); ++y)
        for (int32_t x = i * v.vx; x < min((i + 1) * v.vx, w.W); ++x) {
            const uint32_t node = level0_node(w, x, y);
            const int32_t h0 = node & 0xFF, h1 = (node >> 8) & 0xFF, h2 = (node >> 16) & 0xFF;
            // floor: layers k with k vz <= h0; slab: h1 <= (k+1) vz and k vz <= h2
            int32_t ka = 0, kb = min(h0 / v.vz, nz - 1);
            for (int pass = 0; pass < 2; ++pass) {
                for (int32_t k = ka; k <= kb; ++k) mask[k >> 5] |= 1u << (k & 31);
                if (pass == 0) {
                    if (h2 <= h0) break;  // no slab (node form: slab iff top > floor)
                    ka = max(0, (h1 + v.vz - 1) / v.vz - 1);
                    kb = min(h2 / v.vz, nz - 1);
                }
            }
        }
    const uint32_t xl = (uint32_t)i & 7, yl = (uint32_t)j & 7;
    const uint32_t base_bit = (xl & 1) | ((yl & 1) << 1) | ((xl & 2) << 2) | ((yl & 2) << 3);
    const uint32_t word_xy = ((xl >> 2) << 1) | ((yl >> 2) << 2);
    for (int32_t k = 0; k < nz; k += 2) {  // layers k, k+1: z bit 0 = 0, 1
        const uint32_t zl = (uint32_t)k & 7;
        const uint32_t tile = ((uint32_t)(k >> 3) * v.ty[0] + ((uint32_t)j >> 3)) * v.tx[0] + ((uint32_t)i >> 3);
        const uint32_t wi = word_xy | ((zl >> 1) & 1) | ((zl >> 2) << 3);
        uint32_t *wp = v.words + v.off[0] + tile * 16 + wi;
        const uint32_t b0 = (mask[k >> 5] >> (k & 31)) & 1u;
        const uint32_t b1 = k + 1 < nz ? (mask[(k + 1) >> 5] >> ((k + 1) & 31)) & 1u : 0u;
        const uint32_t set = (b0 << base_bit) | (b1 << (base_bit + 4));
        if (!fresh) atomicAnd(wp, ~((1u << base_bit) | (1u << (base_bit + 4))));
        if (set) atomicOr(wp, set);
    }
}

// Level-l words over the tiles that hold columns [i0, i0+ni) x [j0, j0+nj)
// (every layer): each word's 32 voxels, each the OR of its eight level-(l-1)
// children, stored whole.
__global__ void k_vox_up(const VoxelDev v, int l, int32_t ti0, int32_t tj0, int32_t nti,
                         int32_t ntj) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t ntz = (v.nz[l] + 7) >> 3;
    if (t >= (int64_t)nti * ntj * ntz * 16) return;
    const uint32_t wi = (uint32_t)(t & 15);
    const int64_t tt = t >> 4;
    const int32_t tx = ti0 + (int32_t)(tt % nti), ty = tj0 + (int32_t)((tt / nti) % ntj),
                  tz = (int32_t)(tt / ((int64_t)nti * ntj));
    uint32_t word = 0;
    for (uint32_t bit = 0; bit < 32; ++bit) {
        const uint32_t m = (wi << 5) | bit;
        const int32_t x = tx * 8 + (int32_t)((m & 1) | ((m >> 2) & 2) | ((m >> 4) & 4));
        const int32_t y = ty * 8 + (int32_t)(((m >> 1) & 1) | ((m >> 3) & 2) | ((m >> 5) & 4));
        const int32_t z = tz * 8 + (int32_t)(((m >> 2) & 1) | ((m >> 4) & 2) | ((m >> 6) & 4));
        if (x >= v.nx[l] || y >= v.ny[l] || z >= v.nz[l]) continue;
        bool occ = false;
        for (int c = 0; c < 8 && !occ; ++c) {
            const int32_t cx = 2 * x + (c & 1), cy = 2 * y + ((c >> 1) & 1), cz = 2 * z + (c >> 2);
            if (cx < v.nx[l - 1] && cy < v.ny[l - 1] && cz < v.nz[l - 1])
                occ = vox_occupied(v, l - 1, cx, cy, cz);
        }
        word |= (occ ? 1u : 0u) << bit;
    }
    v.words[v.off[l] + (((uint32_t)tz * v.ty[l] + (uint32_t)ty) * v.tx[l] + (uint32_t)tx) * 16 + wi] = word;
}

__global__ void __launch_bounds__(kVoxThreads) k_vox_trace(const RenderParams p, const VoxelDev v,
                                                           const VoxelParams q) {
    __shared__ VoxLevel s_lv[kVoxMaxLevels];
    __shared__ float s_frac[kVoxFracTable];
    if (threadIdx.x < (unsigned)v.levels) {
        const int l = threadIdx.x;
        s_lv[l] = VoxLevel{v.off[l], v.tx[l], v.ty[l], 0, {v.nx[l], v.ny[l], v.nz[l]}, 0};
    }
    if (threadIdx.x < (unsigned)min(q.inner, kVoxFracTable))
        s_frac[threadIdx.x] = __fdiv_rn(__fadd_rn((float)threadIdx.x, 0.5f), (float)q.inner);
    __syncthreads();
    const CamDev &c = p.cams[blockIdx.y];
    const uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= c.w * c.h) return;
    const int32_t px = (int32_t)(pix % c.w), py = (int32_t)(pix / c.w);
    const int32_t a = 2 * px + 1 - (int32_t)c.w, b = (int32_t)c.h - 1 - 2 * py;
    const float inv_s = 1.0f / 65536.0f;
    float o[3], d[3], inv[3], box[3];
    int32_t vs[3] = {v.vx, v.vy, v.vz};
    const int32_t ve[3] = {pow2_log2(v.vx), pow2_log2(v.vy), pow2_log2(v.vz)};
    for (int k = 0; k < 3; ++k) {
        o[k] = __fmul_rn(__int2float_rn(c.o[k]), inv_s);
        d[k] = __fmul_rn(__int2float_rn(c.F[k] + a * c.R[k] + b * c.U[k]), inv_s);
    }
    box[0] = (float)(v.nx[0] * v.vx);
    box[1] = (float)(v.ny[0] * v.vy);
    box[2] = (float)(v.nz[0] * v.vz);
    const float dl = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                          __fmul_rn(d[2], d[2])));
    float t0 = 0.0f, t1 = __fdiv_rn(q.far_dist, dl);
    bool miss = false;
    for (int k = 0; k < 3; ++k) {
        if (d[k] != 0.0f) {
            inv[k] = __fdiv_rn(1.0f, d[k]);
            const float ta = __fmul_rn(__fsub_rn(0.0f, o[k]), inv[k]);
            const float tb = __fmul_rn(__fsub_rn(box[k], o[k]), inv[k]);
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else {
            inv[k] = 0.0f;
            if (o[k] < 0.0f || o[k] > box[k]) miss = true;
        }
    }
    uint32_t cell = 0xFFFFFFFFu;
    uint8_t layer = 255;
    float depth = __int_as_float(0x7f800000);
    if (!miss && t0 < t1) {
        int l = v.levels - 1;
        float t = t0;
        int ent = -1;
        int32_t idx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float pk = __fadd_rn(o[k], __fmul_rn(d[k], t));
            const float cf = floorf(vox_quot(pk, vs[k], ve[k], l));
            idx[k] = (int32_t)fminf(fmaxf(cf, 0.0f), (float)(s_lv[l].n[k] - 1));
        }
        for (int step = 0; step < q.outer; ++step) {
            float tk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (d[k] != 0.0f) {
                    const float bnd = (float)((idx[k] + (d[k] > 0.0f ? 1 : 0)) * (vs[k] << l));
                    tk[k] = __fmul_rn(__fsub_rn(bnd, o[k]), inv[k]);
                } else {
                    tk[k] = __int_as_float(0x7f800000);
                }
            }
            const float t_out = fminf(fminf(tk[0], tk[1]), tk[2]);
            // a child past the level's end (the last parent of an odd count) is empty
            const VoxLevel &lv = s_lv[l];
            const bool occ = idx[0] < lv.n[0] && idx[1] < lv.n[1] && idx[2] < lv.n[2] &&
                             vox_occupied(v, lv, idx[0], idx[1], idx[2]);
            if (occ && l > 0) {
                --l;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (k == ent) {
                        idx[k] = 2 * idx[k] + (d[k] < 0.0f ? 1 : 0);
                    } else {
                        const float pk = __fadd_rn(o[k], __fmul_rn(d[k], t));
                        const float cf = floorf(vox_quot(pk, vs[k], ve[k], l));
                        idx[k] = (int32_t)fminf(fmaxf(cf, (float)(2 * idx[k])), (float)(2 * idx[k] + 1));
                    }
                }
                continue;
            }
            if (occ) {
                const float span = __fsub_rn(fminf(t_out, t1), t);
                bool found = false;
                for (int s = 0; s < q.inner && !found; ++s) {
                    const float frac = s < kVoxFracTable
                                           ? s_frac[s]
                                           : __fdiv_rn(__fadd_rn((float)s, 0.5f), (float)q.inner);
                    const float ts = __fadd_rn(t, __fmul_rn(span, frac));
                    const float x = __fadd_rn(o[0], __fmul_rn(d[0], ts));
                    const float y = __fadd_rn(o[1], __fmul_rn(d[1], ts));
                    const float z = __fadd_rn(o[2], __fmul_rn(d[2], ts));
                    const float fx = floorf(x), fy = floorf(y);
                    if (!(fx >= 0.0f && fx < (float)p.world.W && fy >= 0.0f && fy < (float)p.world.H))
                        continue;
                    const uint32_t node = level0_node(p.world, (int32_t)fx, (int32_t)fy);
                    const float h0 = (float)(node & 0xFF), h1 = (float)((node >> 8) & 0xFF),
                                h2 = (float)((node >> 16) & 0xFF);
                    const bool fl = z <= h0;
                    const bool up = h2 > h0 && z >= h1 && z <= h2;
                    if (fl || up) {
                        found = true;
                        cell = (uint32_t)fy * (uint32_t)p.world.W + (uint32_t)fx;
                        layer = fl ? 0 : 1;
                        depth = __fmul_rn(ts, dl);
                    }
                }
                if (found) break;
            }
            if (t_out >= t1) break;
            const int ax = tk[0] == t_out ? 0 : (tk[1] == t_out ? 1 : 2);
            const float dax = ax == 0 ? d[0] : (ax == 1 ? d[1] : d[2]);
            const int sg = dax > 0.0f ? 1 : -1;
            int32_t ni;
            if (ax == 0) ni = (idx[0] += sg);
            else if (ax == 1) ni = (idx[1] += sg);
            else ni = (idx[2] += sg);
            t = t_out;
            ent = ax;
            if (ni < 0 || ni >= lv.n[ax]) break;
            if (l < v.levels - 1 && ((ni & 1) == (sg > 0 ? 0 : 1))) {
                ++l;
                idx[0] >>= 1;
                idx[1] >>= 1;
                idx[2] >>= 1;
            }
        }
    }
    if (c.hit_cell) c.hit_cell[pix] = cell;
    if (c.layer) c.layer[pix] = layer;
    if (c.depth) c.depth[pix] = depth;
}

}  // namespace

int voxel_repair(const WorldDev &w, const VoxelDev &v, int32_t x0, int32_t y0, int32_t x1,
                 int32_t y1, bool fresh, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (x1 <= x0 || y1 <= y0) return 0;
    int32_t i0 = x0 / v.vx, i1 = (x1 - 1) / v.vx + 1, j0 = y0 / v.vy, j1 = (y1 - 1) / v.vy + 1;
    {
        const int32_t n = (i1 - i0) * (j1 - j0);
        k_vox_level0<<<(n + 127) / 128, 128, 0, s>>>(w, v, i0, j0, i1 - i0, j1 - j0, fresh ? 1 : 0);
    }
    for (int l = 1; l < v.levels; ++l) {
        i0 >>= 1;
        j0 >>= 1;
        i1 = (i1 + 1) >> 1;
        j1 = (j1 + 1) >> 1;
        const int32_t ti0 = i0 >> 3, tj0 = j0 >> 3, ti1 = (i1 + 7) >> 3, tj1 = (j1 + 7) >> 3;
        const int64_t n = (int64_t)(ti1 - ti0) * (tj1 - tj0) * ((v.nz[l] + 7) >> 3) * 16;
        k_vox_up<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, l, ti0, tj0, ti1 - ti0, tj1 - tj0);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_voxel_trace(const RenderParams &p, const VoxelDev &v, const VoxelParams &q,
                       uint32_t n_cams, uint32_t max_pixels, void *stream) {
    const dim3 grid((max_pixels + kVoxThreads - 1) / kVoxThreads, n_cams);
    k_vox_trace<<<grid, kVoxThreads, 0, (cudaStream_t)stream>>>(p, v, q);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf
