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
// Only suns that rise (Lz > 0), are not vertical and clear the 255-unit
// height range within kSunMaxReach columns have bounds.  An edit of a
// rectangle changes the bounds of cells upstream of it (against L), within the
// distance over which a ray rises by 255 units: sun_bounds_region gives the
// rectangle that holds them, and sun_bounds_repair recomputes, inside it, the
// cells whose bands reach the edited rectangle (a parallelogram along L).
// The band rows and the rise depend on the column of travel only, not on the
// cell: a full build first tabulates them (k_sun_rows) after the bounds words,
// and the build and later repairs read the tables instead of dividing.
#include <cuda_runtime.h>

#include <cstdint>

#include "hf.h"
#include "hf_internal.h"

namespace hf {
namespace {

// Tables after the bounds words, one entry per column of major travel j =
// -1 .. kRowTable - 2 (entry j + 1), all set by one pass per sun:
//   rows:  floor(lmin j / lmaj), the minor-axis rows a ray has crossed;
//   rise:  floor and ceil of 256 j lz / lmaj, its rise in the bounds' units
//          (2^-8 world units), saturated at kRiseSat (every quantity it is
//          compared with is below 2^17, so saturation changes no outcome).
// A bound reads columns up to K + 63 (K <= kSunMaxReach), so every lookup is
// in range; one outside it would fall back to the float-estimated division.
constexpr int kRowTable = (int)kSunMaxReach + 128;
constexpr int32_t kRiseSat = 1 << 21;

__global__ void k_sun_rows(int32_t *q, int64_t lmin, int64_t lmaj, int64_t lz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRowTable) return;
    // once per sun: exact divisions are affordable here
    auto floor_div = [](int64_t n, int64_t d) {
        int64_t f = n / d;
        if (n % d != 0 && n < 0) f -= 1;
        return f;
    };
    const int64_t j = i - 1, rise = 256 * j * lz;
    const int64_t fl = floor_div(rise, lmaj), ce = fl + (fl * lmaj != rise ? 1 : 0);
    q[i] = (int32_t)floor_div(lmin * j, lmaj);
    q[kRowTable + i] = (int32_t)min(fl, (int64_t)kRiseSat);
    q[2 * kRowTable + i] = (int32_t)min(ce, (int64_t)kRiseSat);
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

// floor(a / b) for b > 0 and |a / b| < 2^22: a float estimate, then one
// exact correction (the estimate's relative error is a few 2^-24, so it is
// off by at most one).  Integer division by a run-time 64-bit divisor is a
// long software routine on the GPU; this is a handful of instructions.
__device__ __forceinline__ int64_t floor_div_est(int64_t a, int64_t b, float rcp_b) {
    int64_t q = (int64_t)floorf((float)a * rcp_b);
    const int64_t r = a - q * b;
    if (r < 0) q -= 1;
    else if (r >= b) q += 1;
    return q;
}

// Level-5 node (32 x 32 cells) at major / minor node coordinates.
__device__ __forceinline__ uint32_t node5_at(const WorldDev &w, const SunAxes &a, int32_t nu,
                                             int32_t nv) {
    const int32_t x = a.x_major ? nu : nv, y = a.x_major ? nv : nu;
    return __ldg(w.base + w.off[5] + (uint32_t)y * w.stride[5] + (uint32_t)x);
}

// floor(lmin * j / lmaj) from the rows table.
__device__ __forceinline__ int64_t rows_after(const SunAxes &a, const int32_t *rq, int32_t j,
                                              float rcp_maj) {
    if ((uint32_t)(j + 1) < (uint32_t)kRowTable) return __ldg(rq + j + 1);
    return floor_div_est((int64_t)a.lmin * j, a.lmaj, rcp_maj);
}

// floor (up = false) or ceil (up = true) of 256 j lz / lmaj, j >= 0,
// saturated at kRiseSat, from the rise tables.
__device__ __forceinline__ int32_t rise_after(const SunAxes &a, const int32_t *rq, int32_t j,
                                              bool up, float rcp_maj) {
    if ((uint32_t)(j + 1) < (uint32_t)kRowTable) return __ldg(rq + (up ? 2 : 1) * kRowTable + j + 1);
    const int64_t num = (int64_t)j * 256 * a.lz;
    if (num >= (int64_t)kRiseSat * a.lmaj) return kRiseSat;
    const int64_t f = floor_div_est(num, a.lmaj, rcp_maj);
    return (int32_t)(up && f * a.lmaj != num ? f + 1 : f);
}

// F and G of the cell at major / minor coordinates (cu, cv), rounded to the
// stored units (F down, G up, 2^-8 world units), computed by the 32 lanes of a
// warp: lane l takes column k = k0 + l of each round of 32 (its band's lowest
// floor for F, its widest band's highest top for G), and the warp keeps the
// largest term.  Rounding is monotone, so the largest rounded term is the
// rounded largest term: lanes round first and reduce in 32 bits.  A bound
// stops at the first column it cannot use any more (the grid's end, or for F
// a band that leaves the grid -- monotone in k, so every lane past it is out
// too) or once no later column can raise it.  Where the pyramid has a level
// 5, a round whose region's highest floor (F) or top (G) cannot raise the
// bound loads no cells; the result is the same.
__device__ void bounds_of_warp(const WorldDev &w, const SunAxes &a, const int32_t *rq, int32_t cu,
                               int32_t cv, int32_t NU, int32_t NV, int lane, int32_t &F16,
                               int32_t &G16) {
    const unsigned full = 0xFFFFFFFFu;
    const float rcp_maj = 1.0f / (float)a.lmaj;
    // In the stored units a term is a height h (a floor for F, a top for G)
    // times 256, less the rise 256 (k or k - 1) lz / lmaj: exactly, the F term
    // of column k rounded down is 256 h - ceil(256 k lz / lmaj), and the G term
    // rounded up is 256 h - floor(256 (k - 1) lz / lmaj).  Negative F terms
    // and non-positive G terms never win (F, G >= 0 from k = 0).
    const uint32_t c0 = word_at(w, a, cu, cv);
    F16 = (int32_t)(c0 & 0xFF) << 8;  // k = 0: the start cell's floor
    {  // G, k = 0: the rows the ray can cross in its start column (it moves at
       // most one row there, |lmin| <= lmaj), strictly above: top + 2^-16,
       // rounded up
        const int32_t r0 = cv + (a.lmin < 0 ? -1 : 0), r1 = cv + 1;
        int32_t t = -1;
        if (lane <= r1 - r0) {
            const int32_t r = r0 + lane;
            if (r >= 0 && r < NV) t = (int32_t)((word_at(w, a, cu, r) >> 16) & 0xFF);
        }
        t = __reduce_max_sync(full, t);
        G16 = t < 0 ? 0 : (t << 8) + 1;
    }
    constexpr int32_t top_all = 255 << 8;
    const bool skip = w.L >= 5;
    bool f_on = true, g_on = true;
    for (int32_t k0 = 1;; k0 += 32) {
        // no column from k0 on can raise a bound already this high
        if (f_on && top_all - (F16 + 1) < rise_after(a, rq, k0, true, rcp_maj)) f_on = false;
        if (g_on && top_all - G16 <= rise_after(a, rq, k0 - 1, false, rcp_maj)) g_on = false;
        if (!f_on && !g_on) break;
        const int32_t k = k0 + lane;
        const int32_t col = cu + a.smaj * k;
        const bool in_col = col >= 0 && col < NU;
        // rows floor(lmin * j / lmaj) of travel j = k - 1, k, k + 1
        const int64_t qm = rows_after(a, rq, k - 1, rcp_maj);
        const int64_t qk = rows_after(a, rq, k, rcp_maj);
        const int64_t qp = rows_after(a, rq, k + 1, rcp_maj);
        const int32_t f0 = cv + (int32_t)min(qm, qk), f1 = cv + 1 + (int32_t)max(qm, qk);
        const int32_t g0 = cv + (int32_t)min(qm, qp), g1 = cv + 1 + (int32_t)max(qm, qp);
        const bool f_ok = in_col && f0 >= 0 && f1 < NV;  // the whole F band in the grid
        const bool g_ok = in_col && g1 >= 0 && g0 < NV;  // some of the G band in the grid
        bool f_need = f_on, g_need = g_on;
        if (skip && (f_need || g_need)) {
            // the round's region: its columns and the rows of all its G bands
            const int32_t rlo = max(__reduce_min_sync(full, g_ok ? g0 : 0x7FFFFFFF), 0);
            const int32_t rhi = min(__reduce_max_sync(full, g_ok ? g1 : -1), NV - 1);
            const int32_t ca = cu + a.smaj * k0, cb = cu + a.smaj * (k0 + 31);
            const int32_t clo = max(min(ca, cb), 0), chi = min(max(ca, cb), NU - 1);
            int32_t mh = -1, mt = -1;
            if (rlo <= rhi && clo <= chi) {
                const int32_t nu0 = clo >> 5, nv0 = rlo >> 5;
                const int32_t nnu = (chi >> 5) - nu0 + 1, nnv = (rhi >> 5) - nv0 + 1;
                if (lane < nnu * nnv) {
                    const uint32_t n = node5_at(w, a, nu0 + lane % nnu, nv0 + lane / nnu);
                    mh = (int32_t)(n & 0xFF);
                    mt = (int32_t)((n >> 16) & 0xFF);
                }
                mh = __reduce_max_sync(full, mh);
                mt = __reduce_max_sync(full, mt);
            }
            f_need = f_need && mh >= 0 && (mh << 8) - (F16 + 1) >= rise_after(a, rq, k0, true, rcp_maj);
            g_need = g_need && mt >= 0 && (mt << 8) - G16 > rise_after(a, rq, k0 - 1, false, rcp_maj);
        }
        if (f_need || g_need) {
            int32_t m = 255, t = -1;
            if (g_ok || f_ok)
                for (int32_t r = max(g0, 0); r <= min(g1, NV - 1); ++r) {
                    const uint32_t c = word_at(w, a, col, r);
                    if (r >= f0 && r <= f1) m = min(m, (int32_t)(c & 0xFF));
                    t = max(t, (int32_t)((c >> 16) & 0xFF));
                }
            if (f_need) {
                int32_t v = -1;
                if (f_ok) {
                    const int32_t q = (m << 8) - rise_after(a, rq, k, true, rcp_maj);
                    v = q < 0 ? -1 : q;
                }
                F16 = max(F16, __reduce_max_sync(full, v));
            }
            if (g_need) {
                int32_t v = 0;
                if (g_ok) {
                    const int32_t q = (t << 8) - rise_after(a, rq, k - 1, false, rcp_maj);
                    v = q <= 0 ? 0 : q;
                }
                G16 = max(G16, __reduce_max_sync(full, v));
            }
        }
        if (f_on && !__all_sync(full, f_ok)) f_on = false;
        if (g_on && !__all_sync(full, g_ok)) g_on = false;
    }
}

// Whether the bounds of cell (cu, cv) read any cell of the rectangle
// [eu0, eu1) x [ev0, ev1) (major / minor coordinates): some column of the
// rectangle within `reach` columns downstream, with the cell's widest band
// over those columns meeting the rectangle's rows.
__device__ bool depends_on(const SunAxes &a, const int32_t *rq, int32_t cu, int32_t cv,
                           int32_t eu0, int32_t ev0, int32_t eu1, int32_t ev1, int32_t reach) {
    int32_t ka = a.smaj > 0 ? eu0 - cu : cu - (eu1 - 1);
    int32_t kb = a.smaj > 0 ? eu1 - 1 - cu : cu - eu0;
    ka = max(ka, 0);
    kb = min(kb, reach);
    if (ka > kb) return false;
    // floor is monotone, so the band's lowest and highest rows over the
    // columns ka..kb come from travel ka - 1 and kb + 1
    const float rcp_maj = 1.0f / (float)a.lmaj;
    const int64_t qa = rows_after(a, rq, ka - 1, rcp_maj), qb = rows_after(a, rq, kb + 1, rcp_maj);
    const int32_t r0 = cv + (int32_t)min(qa, qb);
    const int32_t r1 = cv + 1 + (int32_t)max(qa, qb);
    return r1 >= ev0 && r0 < ev1;
}

// One warp per cell of the rectangle [x0, x1) x [y0, y1).  With edit.z >
// edit.x, only the cells whose bounds depend on the edited rectangle
// [edit.x, edit.z) x [edit.y, edit.w) are recomputed (the others keep theirs).
__global__ void k_sun_bounds(const WorldDev w, uint32_t *fg, SunAxes a, int32_t x0, int32_t y0,
                             int32_t nx, uint32_t n, int4 edit, int32_t reach) {
    // the thread index in 64 bits: a warp per cell of a grid of up to 2^28
    // cells is up to 2^33 threads
    const uint32_t i = (uint32_t)(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // warp-uniform
    const int32_t x = x0 + (int32_t)(i % (uint32_t)nx), y = y0 + (int32_t)(i / (uint32_t)nx);
    const int32_t *rq = reinterpret_cast<const int32_t *>(fg + (size_t)w.W * (size_t)w.H);
    if (edit.z > edit.x) {
        const bool dep = a.x_major ? depends_on(a, rq, x, y, edit.x, edit.y, edit.z, edit.w, reach)
                                   : depends_on(a, rq, y, x, edit.y, edit.x, edit.w, edit.z, reach);
        if (!dep) return;  // warp-uniform
    }
    int32_t F16, G16;
    if (a.x_major)
        bounds_of_warp(w, a, rq, x, y, w.W, w.H, lane, F16, G16);
    else
        bounds_of_warp(w, a, rq, y, x, w.H, w.W, lane, F16, G16);
    if (lane == 0)
        fg[(uint32_t)y * (uint32_t)w.W + (uint32_t)x] =
            (uint32_t)max(F16, 0) | ((uint32_t)max(G16, 0) << 16);
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

size_t sun_bounds_bytes(int32_t W, int32_t H) {
    return ((size_t)W * (size_t)H + 3 * (size_t)kRowTable) * sizeof(uint32_t);
}

int sun_bounds(const WorldDev &w, uint32_t *fg, const int32_t sun[3], int32_t x0, int32_t y0,
               int32_t x1, int32_t y1, void *stream) {
    if (!sun_bounds_eligible(sun)) return -1;
    {  // this sun's row and rise tables, which the bounds and later repairs read
        const SunAxes a = axes_of(sun);
        k_sun_rows<<<(kRowTable + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
            reinterpret_cast<int32_t *>(fg + (size_t)w.W * (size_t)w.H), a.lmin, a.lmaj, a.lz);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    if (x1 <= x0 || y1 <= y0) return 0;
    const uint32_t nx = (uint32_t)(x1 - x0), n = nx * (uint32_t)(y1 - y0);
    const uint32_t threads = 128, blocks = (n + threads / 32 - 1) / (threads / 32);
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
    const uint32_t threads = 128, blocks = (n + threads / 32 - 1) / (threads / 32);
    k_sun_bounds<<<blocks, threads, 0, (cudaStream_t)stream>>>(w, fg, a, r[0], r[1], (int32_t)nx,
                                                                n, make_int4(x0, y0, x1, y1),
                                                                reach);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf
