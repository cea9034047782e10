/*
 * hf_oracle.c -- CPU oracle for the two-interval height-field ray cast.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or constant with the CUDA library: every constant below is
 * written out here from the method's definition.
 *
 * What it computes (the plain definition, stepped cell by cell):
 *
 *   A ray is p(t) = O + t d, t >= 0, O in units of 2^-16 world units (S =
 *   65536 per cell / height step), d an integer vector.  The ray visits cell
 *   (i, j) when the set { t >= 0 : (floor(p_x(t)/S), floor(p_y(t)/S)) = (i, j) }
 *   has positive length; each visit has a closed interval [t_in, t_out].
 *   A cell is solid at height z when z <= h0 S, or when it has a slab and
 *   h1 S <= z <= h2 S: the SOLID predicate of the paper's height-field ray
 *   march (Section 3.1), with closed ends and no lower bound on the floor
 *   (the paper's evaluation section records that a z >= 0 guard made height
 *   zero unhittable).  The result is the first visited cell, in visit order,
 *   whose closed interval holds a t with z(t) solid, at the smallest such t;
 *   a miss when the ray leaves the grid first (misses do not manufacture a
 *   ground hit, Section 3.1).
 *
 * Every decision (which cell, which layer, which face) is taken with exact
 * integer arithmetic on __int128; only depth and colour use double.
 * Parity pins: the brute-force per-column checker, closed forms (plane, slab,
 * wall) and invariants in the CPU test suite.
 *
 * Shading is this project's own fixed choice (the paper names palette,
 * diffuse and shadow lookup but gives no constants): an 8-entry albedo table,
 * ambient 0.3 plus diffuse 0.7 times max(0, N.L) times sun visibility, with N
 * the hit face's normal.  Pinned against that stated rule by hand-derived
 * colours for every face, lit, turned away and occluded
 * (tests/golden/shading_faces.json); the paper prints no colours to pin it to.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define OR_S 65536
#define OR_FACE_NX 0
#define OR_FACE_PX 1
#define OR_FACE_NY 2
#define OR_FACE_PY 3
#define OR_FACE_NZ 4
#define OR_FACE_PZ 5
#define OR_FACE_INSIDE 6
#define OR_FACE_MISS 255

/* Rational time t = num / den with den > 0; den == 0 stands for +infinity. */
typedef struct {
    int64_t num, den;
} rat;

static const rat RAT_INF = {1, 0};

static int64_t floor_div(i128 a, int64_t b) /* b > 0 */
{
    i128 q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return (int64_t)q;
}

static int rat_lt(rat a, rat b)
{
    if (a.den == 0) return 0;
    if (b.den == 0) return 1;
    return (i128)a.num * b.den < (i128)b.num * a.den;
}

/* sign(z(t) - level) with z(t) = oz + t dz; at t = +inf the sign of dz rules. */
static int zsign(int64_t oz, int64_t dz, rat t, int64_t level)
{
    if (t.den == 0) {
        if (dz > 0) return 1;
        if (dz < 0) return -1;
        return (oz > level) - (oz < level);
    }
    i128 v = (i128)(oz - level) * t.den + (i128)t.num * dz;
    return (v > 0) - (v < 0);
}

typedef struct {
    int hit;          /* 1 hit, 0 miss */
    int64_t cx, cy;   /* hit cell */
    int layer;        /* 0 floor, 1 slab */
    int face;
    rat t;            /* hit time */
    int64_t steps;    /* cells visited */
} or_hit;

/*
 * Flat exact traversal of one ray over every visited cell.
 * Start cell: floor(O/S) per axis, except that a coordinate lying exactly on
 * a cell boundary with the ray moving toward -axis starts in the lower cell
 * (the cell the ray occupies just after t = 0).
 */
static void trace_ray(const uint32_t *cells, int64_t W, int64_t H,
                      const int64_t o[3], const int64_t d[3], or_hit *r)
{
    r->hit = 0;
    r->cx = r->cy = -1;
    r->layer = 255;
    r->face = OR_FACE_MISS;
    r->t = RAT_INF;
    r->steps = 0;

    int64_t cx = floor_div(o[0], OR_S), cy = floor_div(o[1], OR_S);
    if (d[0] < 0 && cx * OR_S == o[0]) cx -= 1;
    if (d[1] < 0 && cy * OR_S == o[1]) cy -= 1;
    if (cx < 0 || cx >= W || cy < 0 || cy >= H) return;

    rat tin = {0, 1};
    int entry_face = OR_FACE_INSIDE; /* first cell: entered at t = 0 */
    const int64_t oz = o[2], dz = d[2];

    for (;;) {
        r->steps++;
        /* exit time along each axis */
        rat tx = RAT_INF, ty = RAT_INF;
        if (d[0] > 0) tx = (rat){(cx + 1) * OR_S - o[0], d[0]};
        if (d[0] < 0) tx = (rat){o[0] - cx * OR_S, -d[0]};
        if (d[1] > 0) ty = (rat){(cy + 1) * OR_S - o[1], d[1]};
        if (d[1] < 0) ty = (rat){o[1] - cy * OR_S, -d[1]};
        int step_x, step_y;
        rat tout;
        if (tx.den == 0 && ty.den == 0) {
            tout = RAT_INF; step_x = step_y = 0;
        } else if (rat_lt(tx, ty)) {
            tout = tx; step_x = 1; step_y = 0;
        } else if (rat_lt(ty, tx)) {
            tout = ty; step_x = 0; step_y = 1;
        } else { /* exact corner: both axes change at once */
            tout = tx; step_x = step_y = 1;
        }

        uint32_t c = cells[cy * W + cx];
        int64_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF, h2 = (c >> 16) & 0xFF;
        int slab = h1 > h0;

        /* solid at entry? */
        int in_floor = zsign(oz, dz, tin, h0 * OR_S) <= 0;
        int in_slab = slab && zsign(oz, dz, tin, h1 * OR_S) >= 0 &&
                      zsign(oz, dz, tin, h2 * OR_S) <= 0;
        if (in_floor || in_slab) {
            r->hit = 1; r->cx = cx; r->cy = cy;
            r->layer = in_floor ? 0 : 1;
            r->face = entry_face;
            r->t = tin;
            return;
        }
        /* first crossing of a solid boundary inside (t_in, t_out] */
        if (dz < 0) {
            if (slab && zsign(oz, dz, tin, h2 * OR_S) > 0 &&
                zsign(oz, dz, tout, h2 * OR_S) <= 0) {
                r->hit = 1; r->cx = cx; r->cy = cy; r->layer = 1; r->face = OR_FACE_PZ;
                r->t = (rat){oz - h2 * OR_S, -dz};
                return;
            }
            if (zsign(oz, dz, tout, h0 * OR_S) <= 0) {
                r->hit = 1; r->cx = cx; r->cy = cy; r->layer = 0; r->face = OR_FACE_PZ;
                r->t = (rat){oz - h0 * OR_S, -dz};
                return;
            }
        } else if (dz > 0) {
            if (slab && zsign(oz, dz, tin, h1 * OR_S) < 0 &&
                zsign(oz, dz, tout, h1 * OR_S) >= 0) {
                r->hit = 1; r->cx = cx; r->cy = cy; r->layer = 1; r->face = OR_FACE_NZ;
                r->t = (rat){h1 * OR_S - oz, dz};
                return;
            }
        }
        if (!step_x && !step_y) return; /* vertical ray: never leaves its column */
        /* nothing is solid above height 255: a non-descending ray above it misses */
        if (dz >= 0 && zsign(oz, dz, tout, 255 * (int64_t)OR_S) > 0) return;

        if (step_x) {
            cx += d[0] > 0 ? 1 : -1;
            entry_face = d[0] > 0 ? OR_FACE_NX : OR_FACE_PX;
        }
        if (step_y) {
            cy += d[1] > 0 ? 1 : -1;
            if (!step_x) entry_face = d[1] > 0 ? OR_FACE_NY : OR_FACE_PY;
        }
        tin = tout;
        if (cx < 0 || cx >= W || cy < 0 || cy >= H) return;
    }
}

/* ------------------------------------------------------------------ shading */

static const double OR_ALBEDO[8][3] = {
    {0.55, 0.50, 0.40}, {0.35, 0.55, 0.25}, {0.60, 0.60, 0.62}, {0.80, 0.72, 0.50},
    {0.30, 0.30, 0.32}, {0.70, 0.35, 0.20}, {0.90, 0.90, 0.95}, {0.25, 0.40, 0.60},
};
#define OR_KA 0.3
#define OR_KD 0.7
#define OR_SKY 0xFFEBB487u /* r 135, g 180, b 235, a 255 */

static uint32_t shade(uint32_t cell, int face, int visible, const int64_t L[3])
{
    double n = sqrt((double)L[0] * L[0] + (double)L[1] * L[1] + (double)L[2] * L[2]);
    double ndl = 0.0;
    switch (face) {
    case OR_FACE_NX: ndl = -(double)L[0] / n; break;
    case OR_FACE_PX: ndl = (double)L[0] / n; break;
    case OR_FACE_NY: ndl = -(double)L[1] / n; break;
    case OR_FACE_PY: ndl = (double)L[1] / n; break;
    case OR_FACE_NZ: ndl = -(double)L[2] / n; break;
    case OR_FACE_PZ: ndl = (double)L[2] / n; break;
    default: ndl = 0.0;
    }
    if (ndl < 0.0) ndl = 0.0;
    const double *a = OR_ALBEDO[(cell >> 24) & 7];
    double k = OR_KA + OR_KD * ndl * (visible ? 1.0 : 0.0);
    uint32_t out = 0xFF000000u;
    for (int ch = 0; ch < 3; ch++) {
        double v = a[ch] * k;
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        uint32_t q = (uint32_t)floor(255.0 * v + 0.5);
        out |= q << (8 * ch);
    }
    return out;
}

/* Shadow-ray origin: floor of the hit point, then one unit (2^-16) outward
 * along the hit face's normal. */
static void shadow_origin(const int64_t o[3], const int64_t d[3], rat t, int face, int64_t p[3])
{
    for (int i = 0; i < 3; i++) p[i] = o[i] + floor_div((i128)t.num * d[i], t.den);
    switch (face) {
    case OR_FACE_NX: p[0] -= 1; break;
    case OR_FACE_PX: p[0] += 1; break;
    case OR_FACE_NY: p[1] -= 1; break;
    case OR_FACE_PY: p[1] += 1; break;
    case OR_FACE_NZ: p[2] -= 1; break;
    case OR_FACE_PZ: p[2] += 1; break;
    default: break;
    }
}

typedef struct {
    uint32_t *hit_cell;
    uint8_t *layer;
    uint8_t *face;
    double *depth;
    uint32_t *rgba;
    uint8_t *shadow;
    int64_t *steps;
} or_out;

static void ray_full(const uint32_t *cells, int64_t W, int64_t H, const int64_t o[3],
                     const int64_t d[3], const int64_t L[3], int shadows, or_out *out, int64_t k)
{
    or_hit r;
    trace_ray(cells, W, H, o, d, &r);
    if (out->steps) out->steps[k] = r.steps;
    if (!r.hit) {
        out->hit_cell[k] = 0xFFFFFFFFu;
        out->layer[k] = 255;
        out->face[k] = OR_FACE_MISS;
        out->depth[k] = INFINITY;
        out->rgba[k] = OR_SKY;
        if (out->shadow) out->shadow[k] = 0;
        return;
    }
    uint32_t cell = cells[r.cy * W + r.cx];
    out->hit_cell[k] = (uint32_t)(r.cy * W + r.cx);
    out->layer[k] = (uint8_t)r.layer;
    out->face[k] = (uint8_t)r.face;
    double dn = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
    out->depth[k] = ((double)r.t.num / (double)r.t.den) * dn / (double)OR_S;
    int visible = 1;
    if (shadows) {
        if (r.face == OR_FACE_INSIDE) {
            visible = 0;
        } else {
            int64_t p[3];
            or_hit s;
            shadow_origin(o, d, r.t, r.face, p);
            trace_ray(cells, W, H, p, L, &s);
            visible = !s.hit;
        }
        if (out->shadow) out->shadow[k] = (uint8_t)(!visible);
    }
    out->rgba[k] = shade(cell, r.face, visible, L);
}

/* ------------------------------------------------------------ entry points */

typedef struct {
    const uint32_t *cells;
    int64_t W, H;
    const int64_t *cam; /* ox oy oz fx fy fz rx ry rz ux uy uz w h */
    const int64_t *L;
    int shadows;
    int64_t npix;
    const uint32_t *pix; /* NULL: all pixels */
    or_out out;
    int tid, nthreads;
} job;

static void *worker(void *arg)
{
    job *j = (job *)arg;
    const int64_t *c = j->cam;
    int64_t w = c[12], h = c[13];
    const int64_t CH = 64;
    for (int64_t base = (int64_t)j->tid * CH; base < j->npix; base += (int64_t)j->nthreads * CH) {
        int64_t end = base + CH < j->npix ? base + CH : j->npix;
        for (int64_t k = base; k < end; k++) {
            int64_t idx = j->pix ? (int64_t)j->pix[k] : k;
            int64_t px = idx % w, py = idx / w;
            int64_t a = 2 * px + 1 - w, b = h - 1 - 2 * py;
            int64_t d[3];
            for (int i = 0; i < 3; i++) d[i] = c[3 + i] + a * c[6 + i] + b * c[9 + i];
            ray_full(j->cells, j->W, j->H, c, d, j->L, j->shadows, &j->out, k);
        }
    }
    return NULL;
}

/*
 * Render pixels of one camera.  cam = {ox, oy, oz, F, R, U, w, h} (14 int64);
 * pixel (px, py) looks along F + (2px+1-w) R + (h-1-2py) U.  pix lists pixel
 * indices py*w+px (NULL: all w*h pixels, npix must equal w*h); outputs are
 * indexed like pix.  L is the integer sun direction; shadows != 0 traces one
 * shadow ray per hit.  steps (may be NULL) receives the cells visited.
 */
int oracle_render(const uint32_t *cells, int64_t W, int64_t H, const int64_t *cam,
                  const int64_t *L, int shadows, int64_t npix, const uint32_t *pix,
                  uint32_t *hit_cell, uint8_t *layer, uint8_t *face, double *depth,
                  uint32_t *rgba, uint8_t *shadow, int64_t *steps, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) {
        jobs[i] = (job){cells, W, H, cam, L, shadows, npix, pix,
                        {hit_cell, layer, face, depth, rgba, shadow, steps}, i, nthreads};
    }
    for (int i = 1; i < nthreads; i++) pthread_create(&th[i], NULL, worker, &jobs[i]);
    worker(&jobs[0]);
    for (int i = 1; i < nthreads; i++) pthread_join(th[i], NULL);
    return 0;
}

/* Trace n explicit rays (o[3k..3k+2], d[3k..3k+2]); same outputs as above. */
int oracle_trace_rays(const uint32_t *cells, int64_t W, int64_t H, int64_t n,
                      const int64_t *o, const int64_t *d, const int64_t *L, int shadows,
                      uint32_t *hit_cell, uint8_t *layer, uint8_t *face, double *depth,
                      uint32_t *rgba, uint8_t *shadow, int64_t *steps)
{
    or_out out = {hit_cell, layer, face, depth, rgba, shadow, steps};
    for (int64_t k = 0; k < n; k++) ray_full(cells, W, H, o + 3 * k, d + 3 * k, L, shadows, &out, k);
    return 0;
}

/*
 * The min/max pyramid by its definition: node (i, j) of level k >= 1 covers
 * cells [i 2^k, (i+1) 2^k) x [j 2^k, (j+1) 2^k) clipped to the grid and holds
 * byte0 = max h0, byte1 = min over cells of (slab ? h1 : 255),
 * byte2 = max over cells of (slab ? h2 : h0), byte3 = 0.
 * Levels 1..levels are written back to back, level k as ceil(H/2^k) rows of
 * ceil(W/2^k) nodes.  Each node is computed straight from its cells.
 */
int oracle_pyramid(const uint32_t *cells, int64_t W, int64_t H, int levels, uint32_t *out)
{
    int64_t off = 0;
    for (int k = 1; k <= levels; k++) {
        int64_t n = (int64_t)1 << k;
        int64_t wk = (W + n - 1) / n, hk = (H + n - 1) / n;
        for (int64_t j = 0; j < hk; j++) {
            for (int64_t i = 0; i < wk; i++) {
                uint32_t mx0 = 0, mn1 = 255, mxt = 0;
                for (int64_t y = j * n; y < (j + 1) * n && y < H; y++) {
                    for (int64_t x = i * n; x < (i + 1) * n && x < W; x++) {
                        uint32_t c = cells[y * W + x];
                        uint32_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF, h2 = (c >> 16) & 0xFF;
                        int slab = h1 > h0;
                        if (h0 > mx0) mx0 = h0;
                        uint32_t b = slab ? h1 : 255;
                        if (b < mn1) mn1 = b;
                        uint32_t t = slab ? h2 : h0;
                        if (t > mxt) mxt = t;
                    }
                }
                out[off + j * wk + i] = mx0 | (mn1 << 8) | (mxt << 16);
            }
        }
        off += wk * hk;
    }
    return 0;
}
