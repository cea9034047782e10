// hf_trace.cu -- per-pixel exact ray casting through a two-interval height field.
//
// One warp owns one tile of tile_w x tile_h pixels; each lane traces the
// tile's pixels lane, lane+32, ...  Every branch of the traversal is decided
// with exact integer arithmetic on 32-bit operands and 64-bit products, so hit
// cell, layer and face equal the definition bit for bit:
//
//   * ray generation: d = F + (2px+1-w) R + (h-1-2py) U (int32, bounded < 2^21);
//   * times are rationals num/den with 0 <= num <= 2^30 and 0 < den < 2^21;
//   * "z(t) vs h S" is the sign of (oz - hS) den + num dz (|.| < 2^52);
//   * hierarchical DDA over the min/max pyramid: a node whose ray segment lies
//     above its highest top, or above every floor and below every slab
//     underside, is skipped to its exit (the hierarchy may only skip
//     known-empty space, Section 3.2 of the paper); otherwise the traversal
//     descends; at level 0 the cell's two solid intervals are tested (the
//     SOLID predicate of Section 3.1, closed ends, floor unbounded below);
//   * a skip changes only the node index on the exit axis; the finer bits of
//     the other axis are recovered on descent by exact midline tests (no
//     division);
//   * a shadow ray starts at the floor of the hit point (an exact floor
//     division: a float estimate and one integer correction), one fixed-point
//     unit outward along the face normal.
#include <cuda_runtime.h>
#include <math.h>

#include <cstring>
#include <mutex>

#include "hf.h"
#include "hf_internal.h"

namespace hf {
namespace {

#ifndef HF_TRACE_MIN_BLOCKS
#define HF_TRACE_MIN_BLOCKS 3  // resident 256-thread blocks per SM asked of the register allocator (<= 85 registers)
#endif

__constant__ float c_albedo[8][3] = HF_ALBEDO_TABLE;
constexpr float kKa = kAmbient, kKd = kDiffuse;
constexpr uint32_t kSky = kSkyColour;

struct Ray {
    int32_t ox, oy, oz, dx, dy, dz;
};

// One pyramid level as the traversal reads it (a per-block shared table, so
// lanes at different levels read it in one shared-memory access).
struct LevelDev {
    const uint32_t *base;
    uint32_t stride, rows;
};

struct Hit {
    int32_t cx, cy;
    int32_t tnum, tden;  // hit time tnum / tden
    uint32_t word;       // hit cell word
    uint8_t layer, face;
};

struct Counters {
    uint32_t nodes, cells;
};

// sign carrier of z(t) - h S for t = num / den (den > 0):  (oz - hS) den + num dz
__device__ __forceinline__ int64_t zd(int32_t oz_minus_hs, int32_t dz, int32_t num, int32_t den) {
    return (int64_t)oz_minus_hs * den + (int64_t)num * dz;
}

// int64 -> float through two 32-bit conversions (64-bit integer conversions
// run on the FP64 pipe, which is narrow on this GPU).  |v| < 2^52.
__device__ __forceinline__ float i64_to_f32(int64_t v) {
    return fmaf((float)(int32_t)(v >> 32), 4294967296.0f, (float)(uint32_t)v);
}

// floor(a / b) for |a| < 2^52, 0 < b < 2^21 and |a / b| < 2^30: a float
// estimate, a second estimate from the remainder, then one exact correction.
__device__ __forceinline__ int32_t floor_div_small(int64_t a, int32_t b, float rcp_b) {
    int32_t q = (int32_t)floorf(i64_to_f32(a) * rcp_b);        // within ~2^9 of the quotient
    const int32_t r1 = (int32_t)(a - (int64_t)q * b);          // |r1| < 2^31
    q += (int32_t)floorf((float)r1 * rcp_b);                   // within 1
    const int64_t r = a - (int64_t)q * b;
    if (r < 0) q -= 1;
    else if (r >= b) q += 1;
    return q;
}

__device__ __forceinline__ uint32_t load_word(const WorldDev &w, int level, int32_t x, int32_t y) {
    return __ldg(w.base + w.off[level] + (uint32_t)y * w.stride[level] + (uint32_t)x);
}

// Node-form word of level-0 cell (x, y) for the storage the kernel was
// instantiated for (the choice is made at compile time).
template <bool PAIR>
__device__ __forceinline__ uint32_t level0_word(const WorldDev &w, int32_t x, int32_t y) {
    if (PAIR)
        return pair_node(__ldg(w.base + (uint32_t)y * ((uint32_t)w.W >> 1) + ((uint32_t)x >> 1)),
                         (uint32_t)x & 1);
    return load_word(w, 0, x, y);
}

// The two-interval test of one cell over [tin, tout] (tout finite).
// Returns true and fills h on a hit.
__device__ __forceinline__ bool leaf_test(const Ray &r, uint32_t word, int32_t tin_num,
                                          int32_t tin_den, int32_t tout_num, int32_t tout_den,
                                          uint8_t entry_face, Hit &h) {
    const int32_t h0 = word & 0xFF, h1 = (word >> 8) & 0xFF, h2 = (word >> 16) & 0xFF;
    const bool slab = h2 > h0;  // level-0 words are in node form
    const int32_t a0 = r.oz - (h0 << kShift);
    const int64_t zin0 = zd(a0, r.dz, tin_num, tin_den);
    if (zin0 <= 0) {
        h.layer = 0;
        h.face = entry_face;
        h.tnum = tin_num;
        h.tden = tin_den;
        return true;
    }
    const int32_t a1 = r.oz - (h1 << kShift), a2 = r.oz - (h2 << kShift);
    int64_t zin1 = 0, zin2 = 0;
    if (slab) {
        zin1 = zd(a1, r.dz, tin_num, tin_den);
        zin2 = zd(a2, r.dz, tin_num, tin_den);
        if (zin1 >= 0 && zin2 <= 0) {
            h.layer = 1;
            h.face = entry_face;
            h.tnum = tin_num;
            h.tden = tin_den;
            return true;
        }
    }
    if (r.dz < 0) {
        if (slab && zin2 > 0 && zd(a2, r.dz, tout_num, tout_den) <= 0) {
            h.layer = 1;
            h.face = kFacePZ;
            h.tnum = a2;
            h.tden = -r.dz;
            return true;
        }
        if (zd(a0, r.dz, tout_num, tout_den) <= 0) {
            h.layer = 0;
            h.face = kFacePZ;
            h.tnum = a0;
            h.tden = -r.dz;
            return true;
        }
    } else if (r.dz > 0) {
        if (slab && zin1 < 0 && zd(a1, r.dz, tout_num, tout_den) >= 0) {
            h.layer = 1;
            h.face = kFaceNZ;
            h.tnum = -a1;
            h.tden = r.dz;
            return true;
        }
    }
    return false;
}

// A vertical ray (dx = dy = 0) stays in its start column for all t >= 0.
// Writes h only when the ray hits.
__device__ __forceinline__ bool vertical_test(const Ray &r, uint32_t word, Hit &h) {
    const int32_t h0 = word & 0xFF, h1 = (word >> 8) & 0xFF, h2 = (word >> 16) & 0xFF;
    const bool slab = h2 > h0;  // level-0 words are in node form
    const int32_t a0 = r.oz - (h0 << kShift), a1 = r.oz - (h1 << kShift),
                  a2 = r.oz - (h2 << kShift);
    uint8_t layer, face;
    int32_t tnum = 0, tden = 1;
    if (a0 <= 0) {
        layer = 0;
        face = kFaceInside;
    } else if (slab && a1 >= 0 && a2 <= 0) {
        layer = 1;
        face = kFaceInside;
    } else if (r.dz < 0) {
        face = kFacePZ;
        tden = -r.dz;
        layer = (slab && a2 > 0) ? 1 : 0;
        tnum = layer ? a2 : a0;
    } else if (r.dz > 0 && slab && a1 < 0) {
        layer = 1;
        face = kFaceNZ;
        tnum = -a1;
        tden = r.dz;
    } else {
        return false;
    }
    h.layer = layer;
    h.face = face;
    h.tnum = tnum;
    h.tden = tden;
    return true;
}

// Exact first hit of one ray.  h.face = kFaceMiss on a miss, kFaceError when
// max_steps iterations did not finish the ray.
//
// State: the node (nx, ny) at `level` that holds the ray just after t_in.
// Skipping an empty node changes only the node index on the exit axis; the
// finer bits on the other axis are found when the traversal descends, by
// asking whether the ray has crossed the child midline by t_in (exact
// cross-multiplied time comparison).  Every interior cell boundary of a node
// is the midline of exactly one sub-level, so a ray that enters a cell through
// its Y side while also crossing an X cell boundary (a corner) is detected on
// the way down and reported with the X face.
// EMPTY_FIRST picks the order of the two outcomes of the node test in the
// code (empty: advance; else descend or hit); which order runs faster depends
// on the kernel (measured: empty first with shadow rays, the other without).
template <bool STATS, bool PAIR, bool EMPTY_FIRST>
__device__ __forceinline__ void trace_ray(const WorldDev &w, const LevelDev *lvt, const Ray &r,
                                          int start_level, int mip_start, int max_steps, Hit &h,
                                          Counters &cnt) {
    h.face = kFaceMiss;
    h.layer = 255;
    const int32_t adx = abs(r.dx), ady = abs(r.dy);
    int32_t cx = r.ox >> kShift, cy = r.oy >> kShift;
    if (r.dx < 0 && (r.ox & 0xFFFF) == 0) cx -= 1;
    if (r.dy < 0 && (r.oy & 0xFFFF) == 0) cy -= 1;
    if ((uint32_t)cx >= (uint32_t)w.W || (uint32_t)cy >= (uint32_t)w.H) return;

    if (adx == 0 && ady == 0) {
        const uint32_t word = level0_word<PAIR>(w, cx, cy);
        if (STATS) cnt.cells++;
        if (vertical_test(r, word, h)) {
            h.cx = cx;
            h.cy = cy;
            h.word = word;
        }
        return;
    }

    // Per-ray sign constants.  A zero direction component counts as positive:
    // its exit distance is then positive and never the smaller one, so the
    // ray never leaves through that axis.
    const int32_t gx = r.dx < 0 ? -1 : 1, gy = r.dy < 0 ? -1 : 1;  // step per exit
    const int32_t px = r.dx < 0 ? 0 : 1, py = r.dy < 0 ? 0 : 1;    // exit side offset
    const int32_t qx = px ^ 1, qy = py ^ 1;
    const int32_t kx = -gx * r.ox, ky = -gy * r.oy;
    const uint8_t face_x = r.dx < 0 ? kFacePX : kFaceNX;  // entry face of an x crossing
    const uint8_t face_y = r.dy < 0 ? kFacePY : kFaceNY;
    int level = start_level;  // <= mip_start, the coarsest level the ray climbs to
    int32_t nx = cx >> level, ny = cy >> level;
    int32_t tin_num = 0, tin_den = 1;
    uint8_t entry = kFaceInside;


    for (int it = 0;; ++it) {
        // one bounds check per iteration, after every advance, ascent or
        // descent: an index past the level's end, or below 0, means the ray
        // has left the grid.  An ascent keeps the crossed axis out of range
        // (it follows a step onto an even index n >= ceil(E / 2^l), so
        // n / 2 >= ceil(E / 2^(l+1)); or onto -1, and -1 >> 1 = -1).  At an
        // exact corner the other axis may come back in range, in a partial
        // node past the grid's edge; the ray only moves further out, and a
        // descent there lands on an out-of-range child, so it still misses.
        // A ray that leaves on its last allowed iteration is a miss, not a
        // step-limit error.
        const LevelDev lv = lvt[level];
        if ((uint32_t)nx >= lv.stride || (uint32_t)ny >= lv.rows) return;
        if (it == max_steps) break;
        const int32_t bx = (nx + px) << level;  // exit boundary (cells)
        const int32_t by = (ny + py) << level;
        const int32_t numx = gx * (bx << kShift) + kx;  // > 0
        const int32_t numy = gy * (by << kShift) + ky;
        const int64_t cmp = (int64_t)numx * ady - (int64_t)numy * adx;  // < 0: x exits first
        const bool xfirst = cmp <= 0;
        const int32_t tout_num = xfirst ? numx : numy;
        const int32_t tout_den = xfirst ? adx : ady;
        // level 0 holds cells in node form, so one word layout serves every
        // level; for a single cell the emptiness test below is exact (the
        // segment's z range [zlo, zhi] misses (-inf, h0] and [h1, h2] exactly
        // when zlo > top, or zlo > h0 and zhi < h1)
        const uint32_t word =
            PAIR && level == 0
                ? pair_node(__ldg(lv.base + (uint32_t)ny * (lv.stride >> 1) + ((uint32_t)nx >> 1)),
                            (uint32_t)nx & 1)
                : __ldg(lv.base + (uint32_t)ny * lv.stride + (uint32_t)nx);
        const uint32_t node = word;
        if (STATS) {
            if (level > 0) cnt.nodes++;
            else cnt.cells++;
        }
        const int32_t maxh0 = node & 0xFF, minh1 = (node >> 8) & 0xFF,
                      maxtop = (node >> 16) & 0xFF;
        const bool down = r.dz < 0;
        const int32_t lo_num = down ? tout_num : tin_num, lo_den = down ? tout_den : tin_den;
        const int32_t hi_num = down ? tin_num : tout_num, hi_den = down ? tin_den : tout_den;
        const bool empty = zd(r.oz - (maxtop << kShift), r.dz, lo_num, lo_den) > 0 ||
                           (zd(r.oz - (maxh0 << kShift), r.dz, lo_num, lo_den) > 0 &&
                            zd(r.oz - (minh1 << kShift), r.dz, hi_num, hi_den) < 0);
        // advance past the node (or cell) through its exit side; at an exact
        // corner both indices change and the X face is reported
        auto advance = [&]() {
            if (cmp <= 0) nx += gx;
            if (cmp >= 0) ny += gy;
            entry = cmp <= 0 ? face_x : face_y;
            tin_num = tout_num;
            tin_den = tout_den;
            // ascend when the crossed boundary is a parent boundary: the new index
            // on the crossed axis is then even (odd for a negative direction)
            // (as arithmetic, not a branch: one control path for every lane)
            const int32_t crossed = cmp <= 0 ? (nx ^ qx) : (ny ^ qy);
            const int32_t up = (level < mip_start ? 1 : 0) & ~crossed & 1;
            level += up;
            nx >>= up;
            ny >>= up;
        };
        if (EMPTY_FIRST && empty) {
            advance();
            continue;
        }
        if (EMPTY_FIRST || !empty) {
            if (level > 0) {
                // descend into the child that holds the ray just after t_in:
                // the upper child on an axis when the ray has passed that
                // axis' midline by t_in (for a negative direction, when not)
                --level;
                const int32_t xm = (2 * nx + 1) << level, ym = (2 * ny + 1) << level;
                const int64_t lx = (int64_t)(gx * (xm << kShift) + kx) * tin_den;
                const int64_t rx = (int64_t)tin_num * adx;
                const int64_t ly = (int64_t)(gy * (ym << kShift) + ky) * tin_den;
                const int64_t ry = (int64_t)tin_num * ady;
                nx = 2 * nx + ((lx <= rx) != (gx < 0) ? 1 : 0);
                ny = 2 * ny + ((ly <= ry) != (gy < 0) ? 1 : 0);
                // a corner: the ray enters the cell through its Y side and an
                // X cell boundary at the same instant; report the X face
                if (lx == rx && adx != 0 && entry == face_y) entry = face_x;
                continue;
            }
            // a non-empty cell holds the hit (the cell test is exact: the
            // segment's z range meets (-inf, h0] or [h1, h2], and z is
            // continuous along it): find its layer, face and time.  The
            // advance is reached from empty nodes and cells only.
            if (!leaf_test(r, word, tin_num, tin_den, tout_num, tout_den, entry, h)) {
                h.face = kFaceError;  // unreachable: reported, never silent
                h.layer = 255;
                return;
            }
            h.cx = nx;
            h.cy = ny;
            h.word = word;
            return;
        }
        advance();
    }
    h.face = kFaceError;
    h.layer = 255;
}

__device__ __forceinline__ uint32_t shade(uint32_t word, uint8_t face, bool visible,
                                          const float *ln) {
    float ndl;
    switch (face) {
        case kFaceNX: ndl = -ln[0]; break;
        case kFacePX: ndl = ln[0]; break;
        case kFaceNY: ndl = -ln[1]; break;
        case kFacePY: ndl = ln[1]; break;
        case kFaceNZ: ndl = -ln[2]; break;
        case kFacePZ: ndl = ln[2]; break;
        default: ndl = 0.0f;
    }
    const float k = kKa + kKd * fmaxf(ndl, 0.0f) * (visible ? 1.0f : 0.0f);
    const uint32_t m = (word >> 24) & 7;
    uint32_t out = 0xFF000000u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float v = fminf(fmaxf(c_albedo[m][ch] * k, 0.0f), 1.0f);
        out |= ((uint32_t)(255.0f * v + 0.5f)) << (8 * ch);
    }
    return out;
}

// Writes one pixel's outputs.
__device__ __forceinline__ void store_pixel(const RenderParams &p, const CamDev &c, uint32_t pix,
                                            const Hit &ph, float depth, bool visible,
                                            bool shadows) {
    const bool hit = ph.face < kFaceError;
    if (shadows && c.shadow) __stcs(c.shadow + pix, (uint8_t)(visible ? 0 : 1));
    if (c.hit_cell)
        __stcs(c.hit_cell + pix,
               hit ? (uint32_t)ph.cy * (uint32_t)p.world.W + (uint32_t)ph.cx : 0xFFFFFFFFu);
    if (c.layer) __stcs(c.layer + pix, hit ? ph.layer : (uint8_t)255);
    if (c.face) __stcs(c.face + pix, ph.face);
    if (c.depth) __stcs(c.depth + pix, depth);
    if (c.rgba) __stcs(c.rgba + pix, hit ? shade(ph.word, ph.face, visible, p.sun_n) : kSky);
}

// One pixel: its primary ray, then (with shadows) the shadow ray, which
// reuses the same traversal loop and registers.
template <bool SHADOWS, bool STATS, bool PAIR>
__device__ __forceinline__ void trace_pixel(const RenderParams &p, const LevelDev *lvt,
                                            const CamDev &c, int start,
                                            int32_t px, int32_t py, Counters &cnt,
                                            Counters &scnt, uint32_t &nshadow, bool &err) {
    const int32_t a = 2 * px + 1 - (int32_t)c.w;
    const int32_t b = (int32_t)c.h - 1 - 2 * py;
    Ray r;
    r.ox = c.o[0];
    r.oy = c.o[1];
    r.oz = c.o[2];
    r.dx = c.F[0] + a * c.R[0] + b * c.U[0];
    r.dy = c.F[1] + a * c.R[1] + b * c.U[1];
    r.dz = c.F[2] + a * c.R[2] + b * c.U[2];
    Hit ph;  // primary hit, kept while the shadow ray runs
    float depth = __int_as_float(0x7f800000);
    bool visible = true;
    bool shadow_pass = false;
    for (;;) {
        Hit h;
        // one call site: lanes in the primary and in the shadow pass run the
        // same traversal code together
        const bool sp = SHADOWS && shadow_pass;
        Counters pc{0, 0};
        trace_ray<STATS, PAIR, SHADOWS>(p.world, lvt, r, sp ? min(kShadowStart, p.shadow_mip) : start,
                               sp ? p.shadow_mip : p.mip_start, p.max_steps, h, pc);
        if (STATS) {
            Counters &dst = sp ? scnt : cnt;
            dst.nodes += pc.nodes;
            dst.cells += pc.cells;
        }
        if (h.face == kFaceError) err = true;
        if (SHADOWS && shadow_pass) {
            visible = h.face == kFaceMiss;
            break;
        }
        ph = h;
        const bool hit = h.face < kFaceError;
        if (hit) {
            const float fx = (float)r.dx, fy = (float)r.dy, fz = (float)r.dz;
            depth = ((float)h.tnum / (float)h.tden) * sqrtf(fx * fx + fy * fy + fz * fz) *
                    (1.0f / 65536.0f);
        }
        if (!SHADOWS || !hit) break;
        if (h.face == kFaceInside) {
            visible = false;
            break;
        }
        // shadow ray: floor of the hit point, one unit outward along the face normal
        const float rcp_t = 1.0f / (float)h.tden;
        int32_t sxp = r.ox + floor_div_small((int64_t)h.tnum * r.dx, h.tden, rcp_t);
        int32_t syp = r.oy + floor_div_small((int64_t)h.tnum * r.dy, h.tden, rcp_t);
        int32_t szp = r.oz + floor_div_small((int64_t)h.tnum * r.dz, h.tden, rcp_t);
        switch (h.face) {
            case kFaceNX: sxp -= 1; break;
            case kFacePX: sxp += 1; break;
            case kFaceNY: syp -= 1; break;
            case kFacePY: syp += 1; break;
            case kFaceNZ: szp -= 1; break;
            default: szp += 1; break;
        }
        if (STATS) nshadow++;
        if (p.sun_bounds) {
            // the start cell's proven bounds decide most shadow rays at once:
            // at or below F occluded, at or above G lit (hf_sun.cu)
            int32_t bx = sxp >> kShift, by = syp >> kShift;
            if (p.sun[0] < 0 && (sxp & 0xFFFF) == 0) bx -= 1;
            if (p.sun[1] < 0 && (syp & 0xFFFF) == 0) by -= 1;
            if ((uint32_t)bx < (uint32_t)p.world.W && (uint32_t)by < (uint32_t)p.world.H) {
                const uint32_t fg = __ldg(p.sun_bounds + (uint32_t)by * (uint32_t)p.world.W + (uint32_t)bx);
                if (STATS) scnt.cells++;
                if (szp <= (int32_t)((fg & 0xFFFFu) << 8)) {
                    visible = false;
                    break;
                }
                if (szp >= (int32_t)((fg >> 16) << 8)) break;
            }
        }
        r.ox = sxp;
        r.oy = syp;
        r.oz = szp;
        r.dx = p.sun[0];
        r.dy = p.sun[1];
        r.dz = p.sun[2];
        shadow_pass = true;
    }
    store_pixel(p, c, (uint32_t)py * c.w + (uint32_t)px, ph, depth, visible, SHADOWS);
}

// Start level of a camera's primary rays: the largest level l <= mip_start
// whose node around the camera cell has every top below the camera, but not
// below level min(2, mip_start) (a measured floor: climbing out of levels 0
// and 1 costs more steps than the two descents it saves).  Node tops only
// grow with the level, so the levels under the camera are 0..l; lane k tests
// level k.  A camera outside the grid starts at mip_start.  The traversal is
// exact from any start level (a ray climbs as it crosses parent boundaries);
// the rule only saves descents through nodes around the camera that cannot
// be empty.
template <bool PAIR>
__device__ __forceinline__ int primary_start(const RenderParams &p, const CamDev &c, int lane) {
    const WorldDev &w = p.world;
    const int32_t cx = c.o[0] >> kShift, cy = c.o[1] >> kShift;
    if ((uint32_t)cx >= (uint32_t)w.W || (uint32_t)cy >= (uint32_t)w.H) return p.mip_start;
    bool above = false;
    if (lane <= p.mip_start) {
        const uint32_t word =
            lane ? load_word(w, lane, cx >> lane, cy >> lane) : level0_word<PAIR>(w, cx, cy);
        const int32_t top = (word >> 16) & 0xFF;  // every level in node form
        above = c.o[2] > (top << kShift);
    }
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, above);
    return max(min(2, p.mip_start), __ffs(~mask) - 2);
}

// One warp renders one tile: lane l traces the tile's pixels l, l+32, ...
template <bool SHADOWS, bool STATS, bool PAIR>
__device__ __forceinline__ void trace_tile(const RenderParams &p, const LevelDev *lvt,
                                           const CamDev &c, uint32_t local_tile, int lane) {
    const uint32_t tx = local_tile % c.tiles_x, ty = local_tile / c.tiles_x;
    const int32_t tw_log2 = p.tile_w_log2;
    const int32_t x0 = (int32_t)tx << tw_log2, y0 = (int32_t)ty << p.tile_h_log2;
    const int32_t npix = 1 << (tw_log2 + p.tile_h_log2);
    Counters cnt{0, 0}, scnt{0, 0};
    uint32_t nshadow = 0, nrays = 0;
    bool err = false;
    const int start = primary_start<PAIR>(p, c, lane);
    for (int i = lane; i < npix; i += 32) {
        const int32_t px = x0 + (i & ((1 << tw_log2) - 1));
        const int32_t py = y0 + (i >> tw_log2);
        if (px < (int32_t)c.w && py < (int32_t)c.h) {
            trace_pixel<SHADOWS, STATS, PAIR>(p, lvt, c, start, px, py, cnt, scnt, nshadow, err);
            if (STATS) nrays++;
        }
    }
    if (__any_sync(0xFFFFFFFFu, err) && lane == 0) atomicOr(p.status, 1u);
    if (STATS) {
        const uint32_t vn = __reduce_add_sync(0xFFFFFFFFu, cnt.nodes);
        const uint32_t vc = __reduce_add_sync(0xFFFFFFFFu, cnt.cells);
        const uint32_t vr = __reduce_add_sync(0xFFFFFFFFu, nrays);
        const uint32_t vs = __reduce_add_sync(0xFFFFFFFFu, nshadow);
        const uint32_t vf = __reduce_add_sync(0xFFFFFFFFu, scnt.nodes + scnt.cells);
        if (lane == 0) {
            atomicAdd(p.stats + 0, (unsigned long long)vn);
            atomicAdd(p.stats + 1, (unsigned long long)vc);
            atomicAdd(p.stats + 2, (unsigned long long)vr);
            atomicAdd(p.stats + 3, (unsigned long long)vs);
            atomicAdd(p.stats + 4, (unsigned long long)vf);
        }
    }
}

// Asks L2 for the world's coarse levels (all of a small world) as a launch
// starts, spread over all its threads.  A ray's fetches form one dependent
// chain, so a short render of a world that is not in L2 would otherwise wait
// on DRAM at every step of every ray.
__device__ __forceinline__ void prefetch_world(const RenderParams &p) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.prefetch_lines; i += stride)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.prefetch + (size_t)i * 32));
}

// stride of level 0 is its width in cells also for paired texels (whose rows
// then hold stride / 2 words)
__device__ __forceinline__ void fill_levels(LevelDev *s_lv, const WorldDev &w) {
    const int k = threadIdx.x;
    if (k <= w.L) s_lv[k] = LevelDev{w.base + w.off[k], (uint32_t)w.stride[k], (uint32_t)w.rows[k]};
}

// Copy camera i into this warp's shared slot (fields are then read on demand
// instead of being held in registers for the whole tile).
__device__ __forceinline__ const CamDev &stage_cam(CamDev *slot, const CamDev *cams, uint32_t i,
                                                   int lane) {
    static_assert(sizeof(CamDev) % 4 == 0 && sizeof(CamDev) / 4 <= 32, "one word per lane");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(cams + i);
    uint32_t *dst = reinterpret_cast<uint32_t *>(slot);
    __syncwarp();
    if (lane < (int)(sizeof(CamDev) / 4)) dst[lane] = src[lane];
    __syncwarp();
    return *slot;
}

// Persistent batched kernel: warps pop (camera, tile) items from one atomic
// counter until the batch is drained.  One launch renders every camera.
template <bool SHADOWS, bool STATS, bool PAIR>
__global__ void __launch_bounds__(kThreads, HF_TRACE_MIN_BLOCKS) k_trace_batched(const RenderParams p) {
    __shared__ uint32_t s_base[kMaxCams + 1];
    __shared__ CamDev s_cam[kThreads / 32];
    __shared__ LevelDev s_lv[kMaxLevels + 1];
    const uint32_t n = p.hdr->n_cams;
    const uint32_t total = p.hdr->total_tiles;
    prefetch_world(p);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s_base[i] = p.cams[i].tile_base;
    fill_levels(s_lv, p.world);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&p.hdr->counter, 1u);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (t >= total) break;
        // last camera whose first tile is <= t
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_base[mid] <= t) lo = mid;
            else hi = mid;
        }
        const CamDev &c = stage_cam(&s_cam[threadIdx.x >> 5], p.cams, lo, lane);
        trace_tile<SHADOWS, STATS, PAIR>(p, s_lv, c, t - s_base[lo], lane);
    }
}

// Plain kernel: one camera, one warp per tile, grid covers the image once.
// The camera record is a kernel parameter, so a plain render needs no copy of
// it to the device; each warp stages it in shared memory like the batched
// kernel (reading the fields from parameter space instead changes the
// traversal's register allocation, measured 3-8 % slower on large images).
template <bool SHADOWS, bool STATS, bool PAIR>
__global__ void __launch_bounds__(kThreads, HF_TRACE_MIN_BLOCKS)
    k_trace_plain(const __grid_constant__ RenderParams p, const __grid_constant__ CamDev cam,
                  uint32_t n_tiles) {
    __shared__ LevelDev s_lv[kMaxLevels + 1];
    __shared__ CamDev s_cam[kThreads / 32];
    prefetch_world(p);
    fill_levels(s_lv, p.world);
    __syncthreads();
    const uint32_t t = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (t >= n_tiles) return;
    const int lane = threadIdx.x & 31;
    const CamDev &c = stage_cam(&s_cam[threadIdx.x >> 5], &cam, 0, lane);
    trace_tile<SHADOWS, STATS, PAIR>(p, s_lv, c, t, lane);
}

template <bool SH, bool ST, bool PA>
const void *batched_ptr() {
    return reinterpret_cast<const void *>(&k_trace_batched<SH, ST, PA>);
}

template <bool PA>
const void *batched_fn(bool shadows, bool stats) {
    if (shadows) return stats ? batched_ptr<true, true, PA>() : batched_ptr<true, false, PA>();
    return stats ? batched_ptr<false, true, PA>() : batched_ptr<false, false, PA>();
}

template <bool SH, bool ST, bool PA>
void plain_launch(const RenderParams &p, uint32_t blocks, cudaStream_t s, const CamDev &cam,
                  uint32_t n_tiles) {
    k_trace_plain<SH, ST, PA><<<blocks, kThreads, 0, s>>>(p, cam, n_tiles);
}

}  // namespace

const void *trace_batched_fn(bool shadows, bool stats, bool pair) {
    return pair ? batched_fn<true>(shadows, stats) : batched_fn<false>(shadows, stats);
}

int trace_batched_occupancy(bool shadows, bool stats, bool pair, int *blocks_per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, trace_batched_fn(shadows, stats, pair), kThreads, 0);
    return e == cudaSuccess ? 0 : -1;
}

int launch_trace_batched(const RenderParams &p, bool shadows, bool stats, int blocks,
                         void *stream) {
    void *args[] = {const_cast<RenderParams *>(&p)};
    const cudaError_t e =
        cudaLaunchKernel(trace_batched_fn(shadows, stats, p.world.pair != 0), dim3(blocks),
                         dim3(kThreads), args, 0, (cudaStream_t)stream);
    return e == cudaSuccess ? 0 : -1;
}

int launch_trace_plain(const RenderParams &p, bool shadows, bool stats, const CamDev &cam,
                       uint32_t n_tiles, void *stream) {
    if (n_tiles == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t warps = kThreads / 32;
    const uint32_t blocks = (n_tiles + warps - 1) / warps;
    using Fn = void (*)(const RenderParams &, uint32_t, cudaStream_t, const CamDev &, uint32_t);
    static const Fn table[8] = {
        plain_launch<false, false, false>, plain_launch<false, false, true>,
        plain_launch<false, true, false>,  plain_launch<false, true, true>,
        plain_launch<true, false, false>,  plain_launch<true, false, true>,
        plain_launch<true, true, false>,   plain_launch<true, true, true>};
    table[(shadows ? 4 : 0) + (stats ? 2 : 0) + (p.world.pair ? 1 : 0)](p, blocks, s, cam, n_tiles);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf

// ------------------------------------------------------------------------
// Allocation-free render (hf_render_noalloc).  The paper has no counterpart:
// this exists for callers that must not allocate device memory once they are
// running (a render thread whose memory budget is fixed at start-up, or a
// loop where cudaMalloc/cudaFree would stall or implicitly synchronise the
// device).  hf_render may allocate its per-slot camera tables and CUDA graphs
// on first use or when a batch grows; this entry point never does.
//
// Its scratch -- the batch header with the tile counter, the camera table and
// the step-guard status word -- is one file-scope device array, present on
// every GPU that loads this library until the process exits.  Every call
// shares it and it keeps the last call's contents: each call rewrites the
// header (tile counter zero) and the camera table, and clears the status word,
// before its kernel runs.  Two calls whose work overlaps on the GPU race on
// this array; calls ordered on one stream do not.
namespace hf {
namespace {

constexpr size_t kNoallocCamOff = sizeof(BatchHeader);
constexpr size_t kNoallocStatusOff = kNoallocCamOff + (size_t)HF_NOALLOC_MAX_CAMERAS * sizeof(CamDev);
constexpr size_t kNoallocBytes = (kNoallocStatusOff + 64 + 255) & ~(size_t)255;
static_assert(kNoallocStatusOff % 8 == 0, "status words need 8-byte alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device.  In host code the array's name is only a host-side handle.
int noalloc_scratch(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return HF_E_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            (void)cudaGetLastError();
            return HF_E_CUDA;
        }
        g_noalloc_ptr[device] = ptr;
    }
    *out = g_noalloc_ptr[device];
    return HF_OK;
}

int ilog2_pow2(uint32_t v) {
    if (v == 0 || (v & (v - 1))) return -1;
    int k = 0;
    while ((1u << k) < v) ++k;
    return k;
}

}  // namespace
}  // namespace hf

extern "C" int hf_render_noalloc(hf_ctx *ctx, const hf_camera *cams, uint32_t n,
                                 const hf_outputs *outs, const hf_render_opts *opts) {
    using namespace hf;
    if (!ctx) return HF_E_INVALID_ARG;
    if (n == 0) return HF_OK;
    if (!cams || !outs) return HF_E_INVALID_ARG;
    if (n > HF_NOALLOC_MAX_CAMERAS) return HF_E_INVALID_ARG;
    CtxView v;
    if (ctx_view(ctx, &v)) return HF_E_INVALID_ARG;
    hf_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mip_start = HF_MIP_AUTO;
    if (opts) o = *opts;
    if (o.cuda_stream && o.cuda_stream != v.stream) return HF_E_INVALID_ARG;
    // a flag this entry point cannot honour (host outputs, statistics, plain
    // or graph launches, admission) is refused, not silently dropped
    if (o.flags & ~(HF_SHADOWS | HF_SYNC)) return HF_E_INVALID_ARG;
    const uint32_t tw = o.tile_w ? o.tile_w : 8, th = o.tile_h ? o.tile_h : 4;
    const int twl = ilog2_pow2(tw), thl = ilog2_pow2(th);
    if (twl < 0 || thl < 0 || tw * th < 32 || tw * th > 256 || tw > 256 || th > 256)
        return HF_E_INVALID_ARG;
    int32_t sun[3] = {o.sun[0], o.sun[1], o.sun[2]};
    if (sun[0] == 0 && sun[1] == 0 && sun[2] == 0) {
        sun[0] = 321060;
        sun[1] = -321060;
        sun[2] = 262144;
    }
    for (int i = 0; i < 3; ++i)
        if (sun[i] <= -(1 << 21) || sun[i] >= (1 << 21)) return HF_E_INVALID_ARG;

    // header + camera table, built on the stack (no allocation)
    alignas(16) unsigned char buf[kNoallocStatusOff];
    auto *hdr = reinterpret_cast<BatchHeader *>(buf);
    std::memset(hdr, 0, sizeof(*hdr));
    auto *cd = reinterpret_cast<CamDev *>(buf + kNoallocCamOff);
    uint64_t base = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const hf_camera &k = cams[i];
        if (hf_validate_camera((uint32_t)v.world.W, (uint32_t)v.world.H, &k) != HF_OK)
            return HF_E_INVALID_ARG;
        CamDev &c = cd[i];
        for (int a = 0; a < 3; ++a) {
            c.o[a] = (int32_t)k.origin[a];
            c.F[a] = k.fwd[a];
            c.R[a] = k.right[a];
            c.U[a] = k.up[a];
        }
        c.w = k.w;
        c.h = k.h;
        c.tiles_x = (k.w + tw - 1) / tw;
        c.tile_base = (uint32_t)base;
        base += (uint64_t)c.tiles_x * ((k.h + th - 1) / th);
        if (base >= 0xFFFFFFFFull) return HF_E_INVALID_ARG;
        c.hit_cell = outs[i].hit_cell;
        c.layer = outs[i].layer;
        c.face = outs[i].face;
        c.depth = outs[i].depth;
        c.rgba = outs[i].rgba;
        c.shadow = outs[i].shadow;
    }
    hdr->n_cams = n;
    hdr->total_tiles = (uint32_t)base;

    if (cudaSetDevice(v.device) != cudaSuccess) {
        (void)cudaGetLastError();
        return HF_E_CUDA;
    }
    void *scratch = nullptr;
    int rc = noalloc_scratch(v.device, &scratch);
    if (rc != HF_OK) return rc;
    unsigned char *sp = static_cast<unsigned char *>(scratch);
    cudaStream_t stream = (cudaStream_t)v.stream;
    const size_t bytes = kNoallocCamOff + (size_t)n * sizeof(CamDev);
    if (cudaMemcpyAsync(sp, buf, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(sp + kNoallocStatusOff, 0, 64, stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return HF_E_CUDA;
    }
    const bool shadows = (o.flags & HF_SHADOWS) != 0;
    const uint32_t mip = o.mip_start == HF_MIP_AUTO ? kDefaultMipStart : o.mip_start;
    const uint64_t guard = 4ull * ((uint64_t)v.world.W + (uint64_t)v.world.H) + 64;
    const uint32_t steps = o.max_steps ? o.max_steps : (uint32_t)guard;
    if (steps > 0x7FFFFFFFu) return HF_E_INVALID_ARG;
    RenderParams p;
    std::memset(&p, 0, sizeof(p));
    p.world = v.world;
    p.hdr = reinterpret_cast<BatchHeader *>(sp);
    p.cams = reinterpret_cast<const CamDev *>(sp + kNoallocCamOff);
    p.status = reinterpret_cast<uint32_t *>(sp + kNoallocStatusOff);
    p.stats = reinterpret_cast<unsigned long long *>(sp + kNoallocStatusOff + 8);
    p.tile_w_log2 = twl;
    p.tile_h_log2 = thl;
    p.mip_start = (int32_t)(mip > (uint32_t)v.world.L ? (uint32_t)v.world.L : mip);
    p.shadow_mip = (int32_t)((uint32_t)p.mip_start + kShadowMipExtra > (uint32_t)v.world.L
                                 ? (uint32_t)v.world.L
                                 : (uint32_t)p.mip_start + kShadowMipExtra);
    p.max_steps = (int32_t)steps;
    const double sn = sqrt((double)sun[0] * sun[0] + (double)sun[1] * sun[1] +
                           (double)sun[2] * sun[2]);
    for (int i = 0; i < 3; ++i) {
        p.sun[i] = sun[i];
        p.sun_n[i] = (float)(sun[i] / sn);
    }
    const int blocks = v.sm_count * v.occ_shadows[shadows ? 1 : 0];
    if (launch_trace_batched(p, shadows, false, blocks, stream)) return HF_E_CUDA;
    if (o.flags & HF_SYNC) {
        uint32_t status = 0;
        if (cudaMemcpyAsync(&status, p.status, sizeof(status), cudaMemcpyDeviceToHost, stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            (void)cudaGetLastError();
            return HF_E_CUDA;
        }
        if (status) return HF_E_STEP_LIMIT;
    }
    return HF_OK;
}
