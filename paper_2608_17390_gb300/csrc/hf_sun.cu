// hf_sun.cu -- per-cell shadow bounds for one sun direction.
//
// Every shadow ray of a render runs along the same direction L (toward the
// sun), so what it can meet depends only on where it starts.  For each cell c
// two heights bound that in advance, for any origin in c (the cell the ray
// occupies just after t = 0, as the traversal picks it):
//
//   F(c): an origin at height z <= F is occluded.  Let u be the distance the
//         ray has travelled along the major axis of L (the axis with the
//         larger |L| component).  The ray enters the k-th column along that
//         axis after travelling at most k cells, so its height there is at
//         most z + k*Lz/|Lmaj|, and the row it enters lies in a band R_k of at
//         most three rows fixed by c and k.  If that height is at or below the
//         lowest floor of R_k, the cell it enters is solid at its entry time
//         (the floor has no lower bound, Section 3.1): a hit.  F is the best
//         such height over k (k = 0: the start cell's own floor), as long as
//         the band stays inside the grid (a ray that could leave the grid
//         sideways first proves nothing).
//
//   G(c): an origin at height z >= G is lit.  The ray rises, and it is in the
//         k-th column (k >= 1) only after travelling more than k - 1 cells,
//         so its height there exceeds z + (k-1)*Lz/|Lmaj|; every cell it can
//         occupy in that column lies in a band R'_k of at most four rows.  If
//         that bound is at or above every top (the highest solid point of a
//         cell) in R'_k, for every k, nothing is ever solid along the ray.
//
// Both bounds are exact rationals (scaled by |Lmaj|), rounded toward the safe
// side when stored: F down and G up, in units of 2^-8 world units, packed as
// F | G << 16 in one 32-bit word per cell.  A shadow ray whose origin lies at
// or below F is occluded and one at or above G is lit, with no traversal; any
// other is traced as before, so the shadow bit is the same as the flat cast's.
// The shadow map of the paper's shared shading path (Section 3) plays the same
// role -- sun visibility precomputed once per frame -- but approximately;
// these bounds only ever decide cases they prove.
//
// Only suns that rise (Lz > 0) and are not vertical have bounds.  An edit of a
// rectangle changes the bounds of the cells upstream of it (against L) within
// the distance over which a ray can rise by 255 units: sun_bounds_region gives
// that rectangle, and the same kernel recomputes it.
#include <cuda_runtime.h>

#include <cstdint>

#include "hf.h"
#include "hf_internal.h"

namespace hf {
namespace {

constexpr int64_t kS = 1 << kShift;

__device__ __forceinline__ int64_t floor_div64(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

// Node-form word of level-0 cell (x, y), either storage (top = byte 2, floor = byte 0).
__device__ __forceinline__ uint32_t cell_node(const WorldDev &w, int32_t x, int32_t y) {
    return level0_node(w, x, y);
}

struct SunAxes {
    int32_t lmaj;   // |L| along the major axis (> 0)
    int32_t lmin;   // signed L along the minor axis
    int32_t lz;     // > 0
    int32_t smaj;   // +1 / -1: direction along the major axis
    bool x_major;   // the major axis is x
};

__device__ __forceinline__ uint32_t word_at(const WorldDev &w, const SunAxes &a, int32_t cu,
                                            int32_t cv) {
    return a.x_major ? cell_node(w, cu, cv) : cell_node(w, cv, cu);
}

// Level-4 node (16 x 16 cells) at major / minor node coordinates.
__device__ __forceinline__ uint32_t node4_at(const WorldDev &w, const SunAxes &a, int32_t nu,
                                             int32_t nv) {
    const int32_t x = a.x_major ? nu : nv, y = a.x_major ? nv : nu;
    return __ldg(w.base + w.off[4] + (uint32_t)y * w.stride[4] + (uint32_t)x);
}

constexpr int32_t kBlock = 16;  // columns per pyramid-level-4 skip test

// Largest max-floor (byte 0) and max-top (byte 2) over the level-4 nodes
// covering columns cu + smaj*[k, k + kBlock) and the rows every band of those
// columns spans (clipped to the grid).  Returns false when that region lies
// wholly outside the grid along the minor axis.
__device__ bool block_max(const WorldDev &w, const SunAxes &a, int32_t cu, int32_t cv, int32_t k,
                          int32_t NU, int32_t NV, int64_t &maxh0, int64_t &maxtop) {
    const int64_t lmaj = a.lmaj, lmin = a.lmin;
    const int64_t lo = min(lmin * (k - 1), lmin * (k + kBlock)),
                  hi = max(lmin * (k - 1), lmin * (k + kBlock));
    int32_t r0 = cv + (int32_t)floor_div64(lo, lmaj), r1 = cv + 1 + (int32_t)floor_div64(hi, lmaj);
    if (r1 < 0 || r0 >= NV) return false;
    r0 = max(r0, 0);
    r1 = min(r1, NV - 1);
    int32_t c0 = cu + a.smaj * k, c1 = cu + a.smaj * (k + kBlock - 1);
    if (c0 > c1) {
        const int32_t t = c0;
        c0 = c1;
        c1 = t;
    }
    c0 = max(c0, 0);
    c1 = min(c1, NU - 1);
    maxh0 = 0;
    maxtop = 0;
    for (int32_t nu = c0 >> 4; nu <= c1 >> 4; ++nu)
        for (int32_t nv = r0 >> 4; nv <= r1 >> 4; ++nv) {
            const uint32_t n = node4_at(w, a, nu, nv);
            maxh0 = max(maxh0, (int64_t)(n & 0xFF));
            maxtop = max(maxtop, (int64_t)((n >> 16) & 0xFF));
        }
    return true;
}

// F and G of the cell at major / minor coordinates (cu, cv), scaled by lmaj
// (heights in 2^-16 world units times lmaj).  Where the pyramid has a level 4,
// blocks of kBlock columns whose highest floor (for F) or top (for G) cannot
// raise the bound are skipped whole; the result is the same value.
__device__ void bounds_of(const WorldDev &w, const SunAxes &a, int32_t cu, int32_t cv, int32_t NU,
                          int32_t NV, int64_t &F, int64_t &G) {
    const int64_t lmaj = a.lmaj, lmin = a.lmin, lz = a.lz;
    const int64_t top_all = 255 * kS * lmaj;
    const bool skip = w.L >= 4;
    // F: k = 0 is the start cell's floor
    F = (int64_t)(word_at(w, a, cu, cv) & 0xFF) * kS * lmaj;
    for (int32_t k = 1;;) {
        const int32_t col = cu + a.smaj * k;
        if (col < 0 || col >= NU) break;
        const int64_t rise = (int64_t)k * kS * lz;
        if (top_all - rise <= F) break;  // no floor can beat F from here on
        if (skip && (k - 1) % kBlock == 0) {
            int64_t mh, mt;
            if (!block_max(w, a, cu, cv, k, NU, NV, mh, mt)) break;
            if (mh * kS * lmaj - rise <= F) {  // no column of the block can raise F
                k += kBlock;
                continue;
            }
        }
        const int64_t lo = min(lmin * (k - 1), lmin * k), hi = max(lmin * (k - 1), lmin * k);
        const int32_t r0 = cv + (int32_t)floor_div64(lo, lmaj);
        const int32_t r1 = cv + 1 + (int32_t)floor_div64(hi, lmaj);
        if (r0 < 0 || r1 >= NV) break;  // the band drifts out of the grid for good
        int64_t m = 255;
        for (int32_t r = r0; r <= r1; ++r) m = min(m, (int64_t)(word_at(w, a, col, r) & 0xFF));
        F = max(F, m * kS * lmaj - rise);
        ++k;
    }
    // G: k = 0, the rows the ray can cross in its start column, strictly above
    {
        const int32_t r0 = cv + (int32_t)floor_div64(min((int64_t)0, lmin), lmaj);
        const int32_t r1 = cv + 1 + (int32_t)floor_div64(max((int64_t)0, lmin), lmaj);
        G = 0;
        for (int32_t r = max(r0, 0); r <= min(r1, NV - 1); ++r)
            G = max(G, ((int64_t)((word_at(w, a, cu, r) >> 16) & 0xFF) * kS + 1) * lmaj);
    }
    for (int32_t k = 1;;) {
        const int32_t col = cu + a.smaj * k;
        if (col < 0 || col >= NU) break;
        const int64_t rise = (int64_t)(k - 1) * kS * lz;
        if (top_all - rise <= G) break;  // no top can beat G from here on
        if (skip && (k - 1) % kBlock == 0) {
            int64_t mh, mt;
            if (!block_max(w, a, cu, cv, k, NU, NV, mh, mt)) break;
            if (mt * kS * lmaj - rise <= G) {  // no column of the block can raise G
                k += kBlock;
                continue;
            }
        }
        const int64_t lo = min(lmin * (k - 1), lmin * (k + 1)),
                      hi = max(lmin * (k - 1), lmin * (k + 1));
        const int32_t r0 = cv + (int32_t)floor_div64(lo, lmaj);
        const int32_t r1 = cv + 1 + (int32_t)floor_div64(hi, lmaj);
        if (r1 < 0 || r0 >= NV) break;  // the band has left the grid: the ray has too
        int64_t t = -1;
        for (int32_t r = max(r0, 0); r <= min(r1, NV - 1); ++r)
            t = max(t, (int64_t)((word_at(w, a, col, r) >> 16) & 0xFF));
        if (t >= 0) G = max(G, t * kS * lmaj - rise);
        ++k;
    }
}

// Whether the bounds of cell (cu, cv) read any cell of the rectangle
// [eu0, eu1) x [ev0, ev1) (major / minor coordinates): some column of the
// rectangle within `reach` columns downstream, with the cell's widest band
// over those columns meeting the rectangle's rows.
__device__ bool depends_on(const SunAxes &a, int32_t cu, int32_t cv, int32_t eu0, int32_t ev0,
                           int32_t eu1, int32_t ev1, int32_t reach) {
    int32_t ka = a.smaj > 0 ? eu0 - cu : cu - (eu1 - 1);
    int32_t kb = a.smaj > 0 ? eu1 - 1 - cu : cu - eu0;
    ka = max(ka, 0);
    kb = min(kb, reach);
    if (ka > kb) return false;
    const int64_t lmin = a.lmin, lmaj = a.lmaj;
    const int64_t lo = min(lmin * (ka - 1), lmin * (kb + 1)), hi = max(lmin * (ka - 1), lmin * (kb + 1));
    const int32_t r0 = cv + (int32_t)floor_div64(lo, lmaj), r1 = cv + 1 + (int32_t)floor_div64(hi, lmaj);
    return r1 >= ev0 && r0 < ev1;
}

// One thread per cell of the rectangle [x0, x1) x [y0, y1).  With ex1 > ex0,
// only the cells whose bounds depend on the edited rectangle [ex0, ex1) x
// [ey0, ey1) are recomputed (the others keep their words).
__global__ void k_sun_bounds(const WorldDev w, uint32_t *fg, SunAxes a, int32_t x0, int32_t y0,
                             int32_t nx, uint32_t n, int4 edit, int32_t reach) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t x = x0 + (int32_t)(i % (uint32_t)nx), y = y0 + (int32_t)(i / (uint32_t)nx);
    if (edit.z > edit.x) {
        const bool dep = a.x_major ? depends_on(a, x, y, edit.x, edit.y, edit.z, edit.w, reach)
                                   : depends_on(a, y, x, edit.y, edit.x, edit.w, edit.z, reach);
        if (!dep) return;
    }
    int64_t F, G;
    if (a.x_major)
        bounds_of(w, a, x, y, w.W, w.H, F, G);
    else
        bounds_of(w, a, y, x, w.H, w.W, F, G);
    const int64_t unit = (int64_t)a.lmaj << 8;  // 2^-8 world units, unscaled
    int64_t f = floor_div64(F, unit), g = -floor_div64(-G, unit);
    f = f < 0 ? 0 : (f > 65535 ? 65535 : f);
    g = g < 0 ? 0 : (g > 65535 ? 65535 : g);
    fg[(uint32_t)y * (uint32_t)w.W + (uint32_t)x] = (uint32_t)f | ((uint32_t)g << 16);
}

SunAxes axes_of(const int32_t sun[3]) {
    SunAxes a;
    const int32_t ax = sun[0] < 0 ? -sun[0] : sun[0], ay = sun[1] < 0 ? -sun[1] : sun[1];
    a.x_major = ax >= ay;
    a.lmaj = a.x_major ? ax : ay;
    a.lmin = a.x_major ? sun[1] : sun[0];
    a.smaj = (a.x_major ? sun[0] : sun[1]) < 0 ? -1 : 1;
    a.lz = sun[2];
    return a;
}

}  // namespace

bool sun_bounds_eligible(const int32_t sun[3]) {
    if (sun[2] <= 0 || (sun[0] == 0 && sun[1] == 0)) return false;
    const SunAxes a = axes_of(sun);
    // the columns a ray crosses before it has risen by 255 units: the work
    // per cell grows with it, so suns lower than this are traced instead
    return 255 * (int64_t)a.lmaj / a.lz + 2 <= kSunMaxReach;
}

void sun_bounds_region(const WorldDev &w, const int32_t sun[3], int32_t x0, int32_t y0,
                       int32_t x1, int32_t y1, int32_t *out) {
    const SunAxes a = axes_of(sun);
    // beyond K columns a ray has risen past every top: no term there matters
    const int64_t K = 255 * (int64_t)a.lmaj / a.lz + 2;
    const int64_t D = (int64_t)(a.lmin < 0 ? -a.lmin : a.lmin) * (K + 1) / a.lmaj + 2;
    int64_t u0 = a.x_major ? x0 : y0, u1 = a.x_major ? x1 : y1;
    int64_t v0 = a.x_major ? y0 : x0, v1 = a.x_major ? y1 : x1;
    if (a.smaj > 0) u0 -= K;  // upstream: cells whose rays run into the rectangle
    else u1 += K;
    v0 -= D;
    v1 += D;
    const int64_t NU = a.x_major ? w.W : w.H, NV = a.x_major ? w.H : w.W;
    u0 = u0 < 0 ? 0 : u0;
    v0 = v0 < 0 ? 0 : v0;
    u1 = u1 > NU ? NU : u1;
    v1 = v1 > NV ? NV : v1;
    out[0] = (int32_t)(a.x_major ? u0 : v0);
    out[1] = (int32_t)(a.x_major ? v0 : u0);
    out[2] = (int32_t)(a.x_major ? u1 : v1);
    out[3] = (int32_t)(a.x_major ? v1 : u1);
}

int sun_bounds(const WorldDev &w, uint32_t *fg, const int32_t sun[3], int32_t x0, int32_t y0,
               int32_t x1, int32_t y1, void *stream) {
    if (!sun_bounds_eligible(sun)) return -1;
    if (x1 <= x0 || y1 <= y0) return 0;
    const uint32_t nx = (uint32_t)(x1 - x0), n = nx * (uint32_t)(y1 - y0);
    const uint32_t threads = 128, blocks = (n + threads - 1) / threads;
    k_sun_bounds<<<blocks, threads, 0, (cudaStream_t)stream>>>(w, fg, axes_of(sun), x0, y0,
                                                                (int32_t)nx, n,
                                                                make_int4(0, 0, 0, 0), 0);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int sun_bounds_repair(const WorldDev &w, uint32_t *fg, const int32_t sun[3], int32_t x0,
                      int32_t y0, int32_t x1, int32_t y1, void *stream) {
    if (!sun_bounds_eligible(sun)) return -1;
    if (x1 <= x0 || y1 <= y0) return 0;
    int32_t r[4];
    sun_bounds_region(w, sun, x0, y0, x1, y1, r);
    if (r[2] <= r[0] || r[3] <= r[1]) return 0;
    const SunAxes a = axes_of(sun);
    const int32_t reach = (int32_t)(255 * (int64_t)a.lmaj / a.lz + 2);
    const uint32_t nx = (uint32_t)(r[2] - r[0]), n = nx * (uint32_t)(r[3] - r[1]);
    const uint32_t threads = 128, blocks = (n + threads - 1) / threads;
    k_sun_bounds<<<blocks, threads, 0, (cudaStream_t)stream>>>(w, fg, a, r[0], r[1], (int32_t)nx,
                                                                n, make_int4(x0, y0, x1, y1),
                                                                reach);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf
