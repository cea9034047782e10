// hf_api.cpp -- host side of the C ABI declared in include/hf.h.
//
// A context owns one device allocation holding the cells and every pyramid
// level, a pinned staging buffer for edits, and a ring of render slots.  Each
// slot has a pinned camera-table staging buffer, a device copy of it, an event
// that marks the slot's last render as complete, and a small cache of CUDA
// graphs (H2D copy of the camera table -> persistent trace kernel).
//
// Ordering rules (the edit-visibility rule of the paper's Section 4.4):
//   * every edit runs on the context stream, after waiting for the events of
//     all slots, so no in-flight render (on any stream) can observe it;
//   * a render on a foreign stream first waits for the last edit's event.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

namespace {

constexpr int kSlots = 8;
constexpr size_t kScratchAlign = 4096;
constexpr int kMaxGraphsPerSlot = 16;
constexpr int32_t kLimit21 = 1 << 21;
constexpr size_t kPrefetchBytes = 32u << 20;  // world levels warmed in L2 per render launch
constexpr int32_t kDefaultSun[3] = {321060, -321060, 262144};

struct GraphKey {
    uint32_t bytes, shadows, stats, twl, thl, mip, steps;
    int32_t sun[3];
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct Slot {
    void *d_scratch = nullptr;
    void *h_staging = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
    std::vector<std::pair<GraphKey, cudaGraphExec_t>> graphs;
};

}  // namespace

struct hf_ctx {
    int device = 0;
    int sm_count = 0;
    uint32_t W = 0, H = 0, L = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t *d_world = nullptr;
    size_t world_words = 0;
    hf::WorldDev wd{};
    uint32_t *h_edit = nullptr;
    size_t edit_cap = 0;
    cudaEvent_t edit_copy_done = nullptr;
    bool edit_pending = false;
    cudaEvent_t edit_done = nullptr;
    Slot slots[kSlots];
    int next_slot = 0;
    uint32_t *d_status = nullptr;
    uint32_t *h_status = nullptr;
    unsigned long long *d_stats = nullptr;
    int occ[2][2] = {{0, 0}, {0, 0}};
    int occ_march = 0;
    bool pair = false;  // level 0 holds paired 2-byte texels (hf_create_pairs)
    uint32_t *d_sun = nullptr;  // per-cell shadow bounds (hf_sun.cu), allocated on first use
    bool sun_valid = false;     // d_sun holds the bounds of sun_dir for the current cells
    int32_t sun_dir[3] = {0, 0, 0};
    uint32_t *d_vox = nullptr;  // voxel occupancy pyramid (hf_voxel_build), or null
    size_t vox_words = 0;
    hf::VoxelDev vd{};
    // HF_HOST_STAGED: a ring of device staging buffers the chunks render into,
    // the copy stream that streams each finished chunk to the caller's host
    // buffers, and a second render stream (chunks alternate between the
    // caller's stream and it, so one chunk's launch tail overlaps the next)
    char *d_hstage = nullptr;
    size_t hstage_half = 0;  // bytes of one staging buffer
    cudaStream_t copy_stream = nullptr, render2 = nullptr;
    cudaEvent_t stage_ready[4] = {}, stage_free[4] = {}, stage_start = nullptr;
    bool stage_busy[4] = {};
};

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            (void)cudaGetLastError();              \
            return HF_E_CUDA;                      \
        }                                          \
    } while (0)

namespace {

bool cell_ok(uint32_t c) {
    const uint32_t h0 = c & 0xFF, h1 = (c >> 8) & 0xFF, h2 = (c >> 16) & 0xFF;
    if (h1 > h0) return h2 >= h1;
    return h1 == 0 && h2 == 0;
}

// One pair of 2-byte texels (altitude | meta << 8): the pair encoding's rules
// (include/hf.h, hf_create_pairs).
bool pair_ok(uint16_t e, uint16_t o) {
    const uint32_t ve = e & 0xFF, me = e >> 8, vo = o & 0xFF, mo = o >> 8;
    if ((me >> 7) != (mo >> 7)) return false;
    const uint32_t ne = (me >> 3) & 15, no = (mo >> 3) & 15;
    if (!(me >> 7)) return ne == 0 && no == 0;
    const int32_t mid = (int32_t)vo - (int32_t)(16 * ne + no);
    return (int32_t)ve < mid && mid <= (int32_t)vo;
}

int check_pair_rows(const uint16_t *t, uint32_t w, uint32_t h, size_t stride, size_t *bad) {
    if (w % 2) return HF_E_INVALID_ARG;
    for (uint32_t y = 0; y < h; ++y)
        for (uint32_t x = 0; x < w; x += 2)
            if (!pair_ok(t[(size_t)y * stride + x], t[(size_t)y * stride + x + 1])) {
                if (bad) *bad = (size_t)y * w + x;
                return HF_E_INVALID_ARG;
            }
    return HF_OK;
}

// Two valid cell words as one pair of texels; false when the pair encoding
// cannot hold them (one slab without the other, or different slab columns).
bool encode_pair(uint32_t ce, uint32_t co, uint16_t *te, uint16_t *to) {
    const uint32_t e0 = ce & 0xFF, e1 = (ce >> 8) & 0xFF, e2 = (ce >> 16) & 0xFF, em = (ce >> 24) & 7;
    const uint32_t o0 = co & 0xFF, o1 = (co >> 8) & 0xFF, o2 = (co >> 16) & 0xFF, om = (co >> 24) & 7;
    if ((ce >> 27) || (co >> 27)) return false;  // materials above 7 have no room
    const bool se = e1 > e0, so = o1 > o0;
    if (se != so) return false;
    if (!se) {
        *te = (uint16_t)(e0 | (em << 8));
        *to = (uint16_t)(o0 | (om << 8));
        return true;
    }
    if (e0 != o0 || e1 != o1 || e2 != o2) return false;
    const uint32_t delta = e2 - e1;  // 0..254
    *te = (uint16_t)(e0 | ((0x80 | ((delta >> 4) << 3) | em) << 8));
    *to = (uint16_t)(e2 | ((0x80 | ((delta & 15) << 3) | om) << 8));
    return true;
}

int check_rows(const uint32_t *cells, uint32_t w, uint32_t h, size_t stride) {
    for (uint32_t y = 0; y < h; ++y) {
        const uint32_t *row = cells + (size_t)y * stride;
        for (uint32_t x = 0; x < w; ++x)
            if (!cell_ok(row[x])) return HF_E_INVALID_ARG;
    }
    return HF_OK;
}

int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

double rnd(double v) { return std::copysign(std::floor(std::fabs(v) + 0.5), v); }

uint32_t levels_for(uint32_t W, uint32_t H) {
    const uint32_t m = W > H ? W : H;
    uint32_t L = 0;
    while ((1u << L) < m) ++L;
    return L;
}

int ilog2_exact(uint32_t v) {
    if (v == 0 || (v & (v - 1))) return -1;
    int k = 0;
    while ((1u << k) < v) ++k;
    return k;
}

int sync_slots(hf_ctx *c) {
    for (auto &s : c->slots) {
        if (s.pending) {
            CK(cudaEventSynchronize(s.done));
            s.pending = false;
        }
    }
    return HF_OK;
}

void free_graphs(Slot &s) {
    for (auto &g : s.graphs) cudaGraphExecDestroy(g.second);
    s.graphs.clear();
}

int read_status(hf_ctx *c) {
    CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (*c->h_status) {
        CK(cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return HF_E_STEP_LIMIT;
    }
    return HF_OK;
}

}  // namespace

namespace hf {

int ctx_view(const hf_ctx *c, CtxView *out) {
    if (!c || !out) return -1;
    out->world = c->wd;
    out->stream = c->stream;
    out->device = c->device;
    out->sm_count = c->sm_count;
    out->occ_shadows[0] = c->occ[0][0];
    out->occ_shadows[1] = c->occ[1][0];
    return 0;
}

}  // namespace hf

extern "C" {

const char *hf_strerror(int code) {
    switch (code) {
        case HF_OK: return "ok";
        case HF_E_INVALID_ARG: return "invalid argument";
        case HF_E_OUT_OF_BOUNDS: return "rectangle outside the grid";
        case HF_E_OOM: return "out of memory";
        case HF_E_CUDA: return "CUDA runtime error";
        case HF_E_STEP_LIMIT: return "a ray exceeded its traversal step guard";
        case HF_E_BUSY: return "every render slot is in flight";
        default: return "unknown error";
    }
}

int hf_validate_cells(const uint32_t *cells, size_t n, size_t *bad_index) {
    if (!cells && n) return HF_E_INVALID_ARG;
    for (size_t i = 0; i < n; ++i) {
        if (!cell_ok(cells[i])) {
            if (bad_index) *bad_index = i;
            return HF_E_INVALID_ARG;
        }
    }
    return HF_OK;
}

int hf_validate_pairs(const uint16_t *texels, uint32_t width, uint32_t height, size_t row_stride,
                      size_t *bad_index) {
    if ((!texels && width && height) || width % 2) return HF_E_INVALID_ARG;
    const size_t stride = row_stride ? row_stride : width;
    if (stride < width) return HF_E_INVALID_ARG;
    return check_pair_rows(texels, width, height, stride, bad_index);
}

int hf_validate_camera(uint32_t W, uint32_t H, const hf_camera *c) {
    if (!c || W == 0 || H == 0 || W > HF_MAX_DIM || H > HF_MAX_DIM) return HF_E_INVALID_ARG;
    if (c->w == 0 || c->h == 0 || c->w > HF_MAX_DIM || c->h > HF_MAX_DIM) return HF_E_INVALID_ARG;
    if (c->origin[0] < 0 || c->origin[0] >= (int64_t)W << 16) return HF_E_INVALID_ARG;
    if (c->origin[1] < 0 || c->origin[1] >= (int64_t)H << 16) return HF_E_INVALID_ARG;
    if (c->origin[2] < 0 || c->origin[2] >= ((int64_t)1 << 28)) return HF_E_INVALID_ARG;
    for (int i = 0; i < 3; ++i) {
        if (iabs64(c->fwd[i]) >= kLimit21) return HF_E_INVALID_ARG;
        if (iabs64(c->right[i]) * (int64_t)(c->w - 1) >= kLimit21) return HF_E_INVALID_ARG;
        if (iabs64(c->up[i]) * (int64_t)(c->h - 1) >= kLimit21) return HF_E_INVALID_ARG;
        for (int ca = 0; ca < 2; ++ca) {
            for (int cb = 0; cb < 2; ++cb) {
                const int64_t a = ca ? (int64_t)c->w - 1 : 1 - (int64_t)c->w;
                const int64_t b = cb ? (int64_t)c->h - 1 : 1 - (int64_t)c->h;
                const int64_t d = (int64_t)c->fwd[i] + a * c->right[i] + b * c->up[i];
                if (iabs64(d) >= kLimit21) return HF_E_INVALID_ARG;
            }
        }
    }
    return HF_OK;
}

int hf_camera_from_pose(double x, double y, double z, double yaw_deg, double pitch_deg,
                        double hfov_deg, uint32_t w, uint32_t h, hf_camera *out) {
    if (!out || w == 0 || h == 0 || w > HF_MAX_DIM || h > HF_MAX_DIM) return HF_E_INVALID_ARG;
    if (!(hfov_deg > 0.0 && hfov_deg < 180.0)) return HF_E_INVALID_ARG;
    const double deg = M_PI / 180.0;
    const double yaw = yaw_deg * deg, pitch = pitch_deg * deg;
    const double sy = std::sin(yaw), cy = std::cos(yaw), sp = std::sin(pitch),
                 cp = std::cos(pitch);
    const double fwd[3] = {sy * cp, cy * cp, sp};
    const double right[3] = {cy, -sy, 0.0};
    const double up[3] = {-sy * sp, -cy * sp, cp};
    const double f_px = (w / 2.0) / std::tan(hfov_deg * deg / 2.0);
    const double scale = 262144.0 / f_px;
    for (int i = 0; i < 3; ++i) {
        out->fwd[i] = (int32_t)rnd(524288.0 * fwd[i]);
        out->right[i] = (int32_t)rnd(scale * right[i]);
        out->up[i] = (int32_t)rnd(scale * up[i]);
    }
    out->origin[0] = (int64_t)rnd(x * 65536);
    out->origin[1] = (int64_t)rnd(y * 65536);
    out->origin[2] = (int64_t)rnd(z * 65536);
    out->w = w;
    out->h = h;
    return HF_OK;
}

int hf_destroy(hf_ctx *c) {
    if (!c) return HF_OK;
    int rc = HF_OK;
    cudaSetDevice(c->device);
    sync_slots(c);
    if (c->stream && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HF_E_CUDA;
    for (auto &s : c->slots) {
        free_graphs(s);
        if (s.done) cudaEventDestroy(s.done);
        if (s.d_scratch) cudaFree(s.d_scratch);
        if (s.h_staging) cudaFreeHost(s.h_staging);
    }
    if (c->edit_copy_done) cudaEventDestroy(c->edit_copy_done);
    if (c->edit_done) cudaEventDestroy(c->edit_done);
    if (c->h_edit) cudaFreeHost(c->h_edit);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_stats) cudaFree(c->d_stats);
    if (c->d_world) cudaFree(c->d_world);
    if (c->d_vox) cudaFree(c->d_vox);
    if (c->d_sun) cudaFree(c->d_sun);
    if (c->render2) {
        if (cudaStreamSynchronize(c->render2) != cudaSuccess) rc = HF_E_CUDA;
        cudaStreamDestroy(c->render2);
    }
    if (c->copy_stream) {
        if (cudaStreamSynchronize(c->copy_stream) != cudaSuccess) rc = HF_E_CUDA;
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->stage_start) cudaEventDestroy(c->stage_start);
    for (int b = 0; b < 4; ++b) {
        if (c->stage_ready[b]) cudaEventDestroy(c->stage_ready[b]);
        if (c->stage_free[b]) cudaEventDestroy(c->stage_free[b]);
    }
    if (c->d_hstage) cudaFree(c->d_hstage);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    (void)cudaGetLastError();
    delete c;
    return rc;
}

// d->cells holds cell words, or (texels != nullptr) paired 2-byte texels.
static int create_impl(const hf_desc *d, hf_ctx *c, const uint16_t *texels = nullptr) {
    c->pair = texels != nullptr;
    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    c->W = d->width;
    c->H = d->height;
    c->L = levels_for(c->W, c->H);
    if (d->cuda_stream) {
        c->stream = (cudaStream_t)d->cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    // level layout: cells, then each pyramid level, 64-word (256 B) aligned
    size_t off = 0;
    for (uint32_t k = 0; k <= c->L; ++k) {
        const uint32_t wk = (c->W + (1u << k) - 1) >> k, hk = (c->H + (1u << k) - 1) >> k;
        c->wd.off[k] = (uint32_t)off;
        c->wd.stride[k] = wk;
        c->wd.rows[k] = hk;
        const size_t words = (k == 0 && c->pair) ? (size_t)wk / 2 * hk : (size_t)wk * hk;
        off += (words + 63) & ~(size_t)63;
    }
    c->world_words = off;
    c->wd.W = (int32_t)c->W;
    c->wd.H = (int32_t)c->H;
    c->wd.L = (int32_t)c->L;
    c->wd.pair = c->pair ? 1 : 0;
    if (cudaMalloc(&c->d_world, off * sizeof(uint32_t)) != cudaSuccess) {
        (void)cudaGetLastError();
        return HF_E_OOM;
    }
    c->wd.base = c->d_world;
    const size_t stride = d->row_stride ? d->row_stride : d->width;
    if (c->pair) {  // texels are stored as given
        CK(cudaMemcpy2DAsync(c->d_world, (size_t)c->W * 2, texels, stride * 2, (size_t)c->W * 2,
                             c->H, cudaMemcpyHostToDevice, c->stream));
    } else {
        CK(cudaMemcpy2DAsync(c->d_world, (size_t)c->W * 4, d->cells, stride * 4,
                             (size_t)c->W * 4, c->H, cudaMemcpyHostToDevice, c->stream));
        // level 0 is kept in node form (hf::cell_encode)
        if (hf::cells_encode(c->d_world, c->W * c->H, c->stream)) return HF_E_CUDA;
    }
    if (hf::pyramid_build(c->d_world, c->wd, c->stream)) return HF_E_CUDA;
    if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_stats, 5 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaHostAlloc(&c->h_status, sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        return HF_E_OOM;
    }
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream));
    CK(cudaMemsetAsync(c->d_stats, 0, 5 * sizeof(unsigned long long), c->stream));
    CK(cudaEventCreateWithFlags(&c->edit_copy_done, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->edit_done, cudaEventDisableTiming));
    CK(cudaEventRecord(c->edit_done, c->stream));
    for (auto &s : c->slots) CK(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    for (int sh = 0; sh < 2; ++sh)
        for (int st = 0; st < 2; ++st)
            if (hf::trace_batched_occupancy(sh, st, c->pair, &c->occ[sh][st]) ||
                c->occ[sh][st] < 1)
                return HF_E_CUDA;
    if (hf::march_occupancy(&c->occ_march) || c->occ_march < 1) return HF_E_CUDA;
    CK(cudaStreamSynchronize(c->stream));
    return HF_OK;
}

int hf_create(const hf_desc *d, hf_ctx **out) {
    if (!out) return HF_E_INVALID_ARG;
    *out = nullptr;
    if (!d || !d->cells || d->width == 0 || d->height == 0 || d->width > HF_MAX_DIM ||
        d->height > HF_MAX_DIM)
        return HF_E_INVALID_ARG;
    const size_t stride = d->row_stride ? d->row_stride : d->width;
    if (stride < d->width) return HF_E_INVALID_ARG;
    if (check_rows(d->cells, d->width, d->height, stride) != HF_OK) return HF_E_INVALID_ARG;
    hf_ctx *c = new (std::nothrow) hf_ctx();
    if (!c) return HF_E_OOM;
    const int rc = create_impl(d, c);
    if (rc != HF_OK) {
        hf_destroy(c);
        return rc;
    }
    *out = c;
    return HF_OK;
}

int hf_create_pairs(const hf_pair_desc *d, hf_ctx **out) {
    if (!out) return HF_E_INVALID_ARG;
    *out = nullptr;
    if (!d || !d->texels || d->width == 0 || d->height == 0 || d->width > HF_MAX_DIM ||
        d->height > HF_MAX_DIM || d->width % 2)
        return HF_E_INVALID_ARG;
    const size_t stride = d->row_stride ? d->row_stride : d->width;
    if (stride < d->width) return HF_E_INVALID_ARG;
    if (check_pair_rows(d->texels, d->width, d->height, stride, nullptr) != HF_OK)
        return HF_E_INVALID_ARG;
    hf_ctx *c = new (std::nothrow) hf_ctx();
    if (!c) return HF_E_OOM;
    hf_desc cd{};
    cd.width = d->width;
    cd.height = d->height;
    cd.row_stride = d->row_stride;
    cd.cuda_stream = d->cuda_stream;
    const int rc = create_impl(&cd, c, d->texels);
    if (rc != HF_OK) {
        hf_destroy(c);
        return rc;
    }
    *out = c;
    return HF_OK;
}

int hf_info(const hf_ctx *c, hf_info_t *out) {
    if (!c || !out) return HF_E_INVALID_ARG;
    out->width = c->W;
    out->height = c->H;
    out->levels = c->L;
    out->render_slots = kSlots;
    out->cell_bytes = (uint64_t)c->W * c->H * (c->pair ? 2 : 4);
    out->cell_format = c->pair ? HF_CELLS_PAIR16 : HF_CELLS_WORD32;
    out->pyramid_bytes = (uint64_t)(c->world_words - c->wd.off[c->L > 0 ? 1 : 0]) * 4;
    if (c->L == 0) out->pyramid_bytes = 0;
    uint64_t sb = 0;
    for (const auto &s : c->slots) sb += s.cap;
    out->scratch_bytes = sb;
    out->device = c->device;
    out->sm_count = c->sm_count;
    return HF_OK;
}

int hf_edit(hf_ctx *c, uint32_t x0, uint32_t y0, uint32_t w, uint32_t h, const uint32_t *cells,
            size_t row_stride) {
    if (!c) return HF_E_INVALID_ARG;
    if (w == 0 || h == 0) return HF_OK;
    if (!cells) return HF_E_INVALID_ARG;
    if ((uint64_t)x0 + w > c->W || (uint64_t)y0 + h > c->H) return HF_E_OUT_OF_BOUNDS;
    const size_t stride = row_stride ? row_stride : w;
    if (stride < w) return HF_E_INVALID_ARG;
    if (check_rows(cells, w, h, stride) != HF_OK) return HF_E_INVALID_ARG;
    if (c->pair && (x0 % 2 || w % 2)) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    const size_t need = (size_t)w * h * (c->pair ? 2 : 4);
    if (c->edit_pending) {
        CK(cudaEventSynchronize(c->edit_copy_done));
        c->edit_pending = false;
    }
    if (need > c->edit_cap) {
        if (c->h_edit) cudaFreeHost(c->h_edit);
        c->h_edit = nullptr;
        c->edit_cap = 0;
        const size_t cap = (need + kScratchAlign - 1) & ~(kScratchAlign - 1);
        if (cudaHostAlloc(&c->h_edit, cap, cudaHostAllocDefault) != cudaSuccess) {
            (void)cudaGetLastError();
            return HF_E_OOM;
        }
        c->edit_cap = cap;
    }
    if (c->pair) {  // staged as paired texels
        uint16_t *t = reinterpret_cast<uint16_t *>(c->h_edit);
        for (uint32_t y = 0; y < h; ++y) {
            const uint32_t *src = cells + (size_t)y * stride;
            for (uint32_t x = 0; x < w; x += 2)
                if (!encode_pair(src[x], src[x + 1], t + (size_t)y * w + x, t + (size_t)y * w + x + 1))
                    return HF_E_INVALID_ARG;
        }
    } else {
        for (uint32_t y = 0; y < h; ++y) {  // staged in node form (hf::cell_encode)
            const uint32_t *src = cells + (size_t)y * stride;
            uint32_t *dst = c->h_edit + (size_t)y * w;
            for (uint32_t x = 0; x < w; ++x) dst[x] = hf::cell_encode(src[x]);
        }
    }
    // no in-flight render may observe the edit
    for (auto &s : c->slots)
        if (s.pending) CK(cudaStreamWaitEvent(c->stream, s.done, 0));
    const size_t cb = c->pair ? 2 : 4;  // bytes per cell at level 0
    CK(cudaMemcpy2DAsync(reinterpret_cast<char *>(c->d_world) + ((size_t)y0 * c->W + x0) * cb,
                         (size_t)c->W * cb, c->h_edit, (size_t)w * cb, (size_t)w * cb, h,
                         cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->edit_copy_done, c->stream));
    c->edit_pending = true;
    if (hf::pyramid_repair(c->d_world, c->wd, (int32_t)x0, (int32_t)y0, (int32_t)(x0 + w),
                           (int32_t)(y0 + h), c->stream))
        return HF_E_CUDA;
    if (c->d_vox && hf::voxel_repair(c->wd, c->vd, (int32_t)x0, (int32_t)y0, (int32_t)(x0 + w),
                                     (int32_t)(y0 + h), false, c->stream))
        return HF_E_CUDA;
    if (c->sun_valid) {  // the shadow bounds of the cells upstream of the rectangle
        if (hf::sun_bounds_repair(c->wd, c->d_sun, c->sun_dir, (int32_t)x0, (int32_t)y0,
                                  (int32_t)(x0 + w), (int32_t)(y0 + h), c->stream)) {
            c->sun_valid = false;
            return HF_E_CUDA;
        }
    }
    CK(cudaEventRecord(c->edit_done, c->stream));
    return HF_OK;
}

int hf_rebuild(hf_ctx *c) {
    if (!c) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    for (auto &s : c->slots)
        if (s.pending) CK(cudaStreamWaitEvent(c->stream, s.done, 0));
    if (hf::pyramid_build(c->d_world, c->wd, c->stream)) return HF_E_CUDA;
    if (c->d_vox) {
        CK(cudaMemsetAsync(c->d_vox, 0, c->vox_words * 4, c->stream));
        if (hf::voxel_repair(c->wd, c->vd, 0, 0, (int32_t)c->W, (int32_t)c->H, true, c->stream))
            return HF_E_CUDA;
    }
    if (c->sun_valid &&
        hf::sun_bounds(c->wd, c->d_sun, c->sun_dir, 0, 0, (int32_t)c->W, (int32_t)c->H, c->stream)) {
        c->sun_valid = false;
        return HF_E_CUDA;
    }
    CK(cudaEventRecord(c->edit_done, c->stream));
    return HF_OK;
}

int hf_sync(hf_ctx *c) {
    if (!c) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    if (sync_slots(c) != HF_OK) return HF_E_CUDA;
    CK(cudaStreamSynchronize(c->stream));
    return read_status(c);
}

int hf_read_cells(hf_ctx *c, uint32_t x0, uint32_t y0, uint32_t w, uint32_t h, uint32_t *out,
                  size_t row_stride) {
    if (!c || !out) return HF_E_INVALID_ARG;
    if (w == 0 || h == 0) return HF_OK;
    if ((uint64_t)x0 + w > c->W || (uint64_t)y0 + h > c->H) return HF_E_OUT_OF_BOUNDS;
    const size_t stride = row_stride ? row_stride : w;
    if (stride < w) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    if (c->pair) {  // the whole pairs that cover the columns, decoded here
        const uint32_t xa = x0 & ~1u, xb = (x0 + w + 1) & ~1u;
        std::vector<uint32_t> pw((size_t)(xb - xa) / 2 * h);
        CK(cudaMemcpy2DAsync(pw.data(), (size_t)(xb - xa) * 2,
                             reinterpret_cast<const char *>(c->d_world) + ((size_t)y0 * c->W + xa) * 2,
                             (size_t)c->W * 2, (size_t)(xb - xa) * 2, h, cudaMemcpyDeviceToHost,
                             c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (uint32_t y = 0; y < h; ++y)
            for (uint32_t x = 0; x < w; ++x) {
                const uint32_t cx = x0 + x;
                out[(size_t)y * stride + x] = hf::cell_decode(
                    hf::pair_node(pw[(size_t)y * ((xb - xa) / 2) + (cx - xa) / 2], cx & 1));
            }
        return HF_OK;
    }
    CK(cudaMemcpy2DAsync(out, stride * 4, c->d_world + (size_t)y0 * c->W + x0, (size_t)c->W * 4,
                         (size_t)w * 4, h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (uint32_t y = 0; y < h; ++y) {  // back from node form
        uint32_t *row = out + (size_t)y * stride;
        for (uint32_t x = 0; x < w; ++x) row[x] = hf::cell_decode(row[x]);
    }
    return HF_OK;
}

int hf_read_pyramid(hf_ctx *c, uint32_t level, uint32_t *out) {
    if (!c || !out || level == 0 || level > c->L) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    const size_t wk = c->wd.stride[level];
    const size_t hk = (c->H + (1u << level) - 1) >> level;
    CK(cudaMemcpyAsync(out, c->d_world + c->wd.off[level], wk * hk * 4, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HF_OK;
}

int hf_read_sun_bounds(hf_ctx *c, uint32_t *out, int32_t sun[3]) {
    if (!c) return HF_E_INVALID_ARG;
    if (!c->sun_valid) return HF_E_INVALID_ARG;
    if (sun)
        for (int i = 0; i < 3; ++i) sun[i] = c->sun_dir[i];
    if (!out) return HF_OK;
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(out, c->d_sun, (size_t)c->W * c->H * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HF_OK;
}

int hf_stats(hf_ctx *c, uint64_t out[5]) {
    if (!c || !out) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    if (sync_slots(c) != HF_OK) return HF_E_CUDA;
    unsigned long long v[5];
    CK(cudaMemcpyAsync(v, c->d_stats, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemsetAsync(c->d_stats, 0, sizeof(v), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 5; ++i) out[i] = v[i];
    return HF_OK;
}

// The shadow bounds of `sun` for the current cells, built on the context's
// stream when the sun differs from the last one (or after a failure); renders
// issued later wait for it like for an edit.  Suns without bounds (not
// rising, vertical, or too low: hf::sun_bounds_eligible) give null.
static int ensure_sun_bounds(hf_ctx *c, const int32_t sun[3], const uint32_t **out) {
    *out = nullptr;
    if (!hf::sun_bounds_eligible(sun)) return HF_OK;
    if (c->sun_valid && std::memcmp(c->sun_dir, sun, sizeof(c->sun_dir)) == 0) {
        *out = c->d_sun;
        return HF_OK;
    }
    CK(cudaSetDevice(c->device));
    if (!c->d_sun) {
        if (cudaMalloc(&c->d_sun, hf::sun_bounds_bytes((int32_t)c->W, (int32_t)c->H)) != cudaSuccess) {
            (void)cudaGetLastError();
            c->d_sun = nullptr;
            return HF_E_OOM;
        }
    }
    // no render in flight may read bounds of another sun while they change
    for (auto &s : c->slots)
        if (s.pending) CK(cudaStreamWaitEvent(c->stream, s.done, 0));
    c->sun_valid = false;
    if (hf::sun_bounds(c->wd, c->d_sun, sun, 0, 0, (int32_t)c->W, (int32_t)c->H, c->stream))
        return HF_E_CUDA;
    CK(cudaEventRecord(c->edit_done, c->stream));
    std::memcpy(c->sun_dir, sun, sizeof(c->sun_dir));
    c->sun_valid = true;
    *out = c->d_sun;
    return HF_OK;
}

static int acquire_slot(hf_ctx *c, bool nowait, int *idx) {
    for (int k = 0; k < kSlots; ++k) {
        const int i = (c->next_slot + k) % kSlots;
        Slot &s = c->slots[i];
        if (!s.pending) {
            *idx = i;
            c->next_slot = (i + 1) % kSlots;
            return HF_OK;
        }
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaSuccess) {
            s.pending = false;
            *idx = i;
            c->next_slot = (i + 1) % kSlots;
            return HF_OK;
        }
        if (q != cudaErrorNotReady) {
            (void)cudaGetLastError();
            return HF_E_CUDA;
        }
    }
    if (nowait) return HF_E_BUSY;
    const int i = c->next_slot;
    CK(cudaEventSynchronize(c->slots[i].done));
    c->slots[i].pending = false;
    *idx = i;
    c->next_slot = (i + 1) % kSlots;
    return HF_OK;
}

static int ensure_slot_cap(Slot &s, size_t bytes) {
    if (bytes <= s.cap) return HF_OK;
    free_graphs(s);
    if (s.d_scratch) cudaFree(s.d_scratch);
    if (s.h_staging) cudaFreeHost(s.h_staging);
    s.d_scratch = nullptr;
    s.h_staging = nullptr;
    s.cap = 0;
    if (cudaMalloc(&s.d_scratch, bytes) != cudaSuccess ||
        cudaHostAlloc(&s.h_staging, bytes, cudaHostAllocDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        return HF_E_OOM;
    }
    s.cap = bytes;
    return HF_OK;
}

static int launch_graph(hf_ctx *c, Slot &s, const GraphKey &key, const hf::RenderParams &p,
                        bool shadows, bool stats, cudaStream_t stream) {
    cudaGraphExec_t exec = nullptr;
    for (auto &g : s.graphs)
        if (g.first == key) exec = g.second;
    if (!exec) {
        cudaGraph_t graph;
        CK(cudaGraphCreate(&graph, 0));
        cudaGraphNode_t copy, kern;
        if (cudaGraphAddMemcpyNode1D(&copy, graph, nullptr, 0, s.d_scratch, s.h_staging, key.bytes,
                                     cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return HF_E_CUDA;
        }
        hf::RenderParams pc = p;
        void *args[] = {&pc};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(hf::trace_batched_fn(shadows, stats, c->pair));
        kp.gridDim = dim3((unsigned)(c->sm_count * c->occ[shadows][stats]));
        kp.blockDim = dim3(hf::kThreads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        if (cudaGraphAddKernelNode(&kern, graph, &copy, 1, &kp) != cudaSuccess ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaGraphDestroy(graph);
            return HF_E_CUDA;
        }
        cudaGraphDestroy(graph);
        if ((int)s.graphs.size() >= kMaxGraphsPerSlot) {
            cudaGraphExecDestroy(s.graphs.front().second);
            s.graphs.erase(s.graphs.begin());
        }
        s.graphs.push_back({key, exec});
    }
    CK(cudaGraphLaunch(exec, stream));
    return HF_OK;
}

// Validates the cameras, takes a render slot and fills its camera table.
struct Batch {
    int slot;
    size_t bytes, bucket;
    std::vector<uint32_t> tiles;
    hf::RenderParams p;
    cudaStream_t stream;
};

// A pinned host buffer's device alias (device memory passes unchanged);
// nullptr for memory the GPU cannot address (pageable or unknown).
static void *device_alias(void *ptr) {
    if (!ptr) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

static int prepare_batch(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                         uint32_t tw, uint32_t th, bool nowait, void *user_stream, Batch &b,
                         bool host_outputs = false, size_t extra_bytes = 0) {
    const int twl = ilog2_exact(tw), thl = ilog2_exact(th);
    if (twl < 0 || thl < 0 || tw * th < 32 || tw * th > 256 || tw > 256 || th > 256)
        return HF_E_INVALID_ARG;
    uint64_t total_tiles = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (hf_validate_camera(c->W, c->H, &cams[i]) != HF_OK) return HF_E_INVALID_ARG;
        const uint64_t tx = (cams[i].w + tw - 1) / tw, ty = (cams[i].h + th - 1) / th;
        total_tiles += tx * ty;
    }
    if (total_tiles >= 0xFFFFFFFFull) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    b.stream = user_stream ? (cudaStream_t)user_stream : c->stream;
    int rc = acquire_slot(c, nowait, &b.slot);
    if (rc != HF_OK) return rc;
    Slot &s = c->slots[b.slot];
    b.bytes = sizeof(hf::BatchHeader) + (size_t)n * sizeof(hf::CamDev) + extra_bytes;
    b.bucket = (b.bytes + kScratchAlign - 1) & ~(kScratchAlign - 1);
    rc = ensure_slot_cap(s, b.bucket);
    if (rc != HF_OK) return rc;
    auto *hdr = (hf::BatchHeader *)s.h_staging;
    std::memset(hdr, 0, sizeof(*hdr));
    hdr->n_cams = n;
    hdr->total_tiles = (uint32_t)total_tiles;
    auto *cd = (hf::CamDev *)((char *)s.h_staging + sizeof(hf::BatchHeader));
    b.tiles.assign(n, 0);
    uint32_t base = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const hf_camera &k = cams[i];
        hf::CamDev &v = cd[i];
        for (int a = 0; a < 3; ++a) {
            v.o[a] = (int32_t)k.origin[a];
            v.F[a] = k.fwd[a];
            v.R[a] = k.right[a];
            v.U[a] = k.up[a];
        }
        v.w = k.w;
        v.h = k.h;
        v.tiles_x = (k.w + tw - 1) / tw;
        b.tiles[i] = v.tiles_x * ((k.h + th - 1) / th);
        v.tile_base = base;
        base += b.tiles[i];
        v.hit_cell = outs[i].hit_cell;
        v.layer = outs[i].layer;
        v.face = outs[i].face;
        v.depth = outs[i].depth;
        v.rgba = outs[i].rgba;
        v.shadow = outs[i].shadow;
        if (host_outputs) {
            const hf_outputs &u = outs[i];
            v.hit_cell = static_cast<uint32_t *>(device_alias(u.hit_cell));
            v.layer = static_cast<uint8_t *>(device_alias(u.layer));
            v.face = static_cast<uint8_t *>(device_alias(u.face));
            v.depth = static_cast<float *>(device_alias(u.depth));
            v.rgba = static_cast<uint32_t *>(device_alias(u.rgba));
            v.shadow = static_cast<uint8_t *>(device_alias(u.shadow));
            if ((u.hit_cell && !v.hit_cell) || (u.layer && !v.layer) || (u.face && !v.face) ||
                (u.depth && !v.depth) || (u.rgba && !v.rgba) || (u.shadow && !v.shadow))
                return HF_E_INVALID_ARG;  // the slot was not yet marked in flight
        }
    }
    std::memset(&b.p, 0, sizeof(b.p));
    b.p.world = c->wd;
    {  // the levels the trace kernels warm in L2: from the finest level whose
       // tail of the world fits kPrefetchBytes (the whole of a small world)
        uint32_t k = 0;
        while (k < (uint32_t)c->L && (c->world_words - c->wd.off[k]) * 4 > kPrefetchBytes) ++k;
        b.p.prefetch = c->wd.base + c->wd.off[k];
        b.p.prefetch_lines = (uint32_t)(((c->world_words - c->wd.off[k]) * 4 + 127) / 128);
    }
    b.p.hdr = (hf::BatchHeader *)s.d_scratch;
    b.p.cams = (const hf::CamDev *)((char *)s.d_scratch + sizeof(hf::BatchHeader));
    b.p.status = c->d_status;
    b.p.stats = c->d_stats;
    b.p.tile_w_log2 = twl;
    b.p.tile_h_log2 = thl;
    if (b.stream != c->stream) CK(cudaStreamWaitEvent(b.stream, c->edit_done, 0));
    return HF_OK;
}

static int finish_batch(hf_ctx *c, Batch &b, bool sync) {
    Slot &s = c->slots[b.slot];
    CK(cudaEventRecord(s.done, b.stream));
    s.pending = true;
    if (sync) {
        CK(cudaEventSynchronize(s.done));
        s.pending = false;
        return read_status(c);
    }
    return HF_OK;
}

// HF_HOST_STAGED: render the cameras in kStageChunks chunks of equal pixel
// counts (no smaller than kMinChunkPx, as each chunk costs a launch and a few
// copies) into a ring of kBuffers device staging buffers, and stream each
// finished chunk to the caller's pinned host buffers on the copy stream while
// later chunks render.  The render stream waits for the last copies.
//
// A chunk is a run of pieces: row bands of the cameras, in order.  Rows
// [row0, row0 + rows) of a camera form a camera of their own, with the same
// origin, right and up vectors, `rows` rows, and fwd moved to the band's
// middle row,
//   fwd' = fwd + (h - rows - 2 row0) up,
// so that each of its pixels has the same integer direction, and therefore
// the same result, as in the whole camera.  fwd' lies between fwd - (h-1) up
// and fwd + (h-1) up, each the mean of two corner directions, so the band is
// valid whenever the camera is.  So one large camera streams too: its copies
// start after its first band.
static int render_host_staged(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                              const hf_render_opts &o) {
#ifndef HF_STAGE_CHUNKS
#define HF_STAGE_CHUNKS 24  // measured: 8 / 12 / 16 / 24 / 32 / 48 / 96 / 192 chunks
#endif
#ifndef HF_STAGE_BUFFERS
#define HF_STAGE_BUFFERS 4  // measured: 2 / 3 / 4 buffers
#endif
    constexpr uint32_t kStageChunks = HF_STAGE_CHUNKS;
    constexpr uint64_t kMinChunkPx = 1u << 19;  // ~40 us of render or copy
    constexpr int kBuffers = HF_STAGE_BUFFERS;
    constexpr size_t kAlign = 256;
    const bool shadows = (o.flags & HF_SHADOWS) != 0;
    // the fields to move, with their element sizes
    auto field_bytes = [&](const hf_outputs &u, int f) -> size_t {
        switch (f) {
            case 0: return u.hit_cell ? 4 : 0;
            case 1: return u.layer ? 1 : 0;
            case 2: return u.face ? 1 : 0;
            case 3: return u.depth ? 4 : 0;
            case 4: return u.rgba ? 4 : 0;
            default: return (u.shadow && shadows) ? 1 : 0;
        }
    };
    auto field_ptr = [](const hf_outputs &u, int f) -> void * {
        switch (f) {
            case 0: return u.hit_cell;
            case 1: return u.layer;
            case 2: return u.face;
            case 3: return u.depth;
            case 4: return u.rgba;
            default: return u.shadow;
        }
    };
    uint64_t total_px = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (hf_validate_camera(c->W, c->H, &cams[i]) != HF_OK) return HF_E_INVALID_ARG;
        total_px += (uint64_t)cams[i].w * cams[i].h;
        for (int f = 0; f < 6; ++f) {
            void *ptr = field_ptr(outs[i], f);
            if (!ptr) continue;
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
                (void)cudaGetLastError();
                return HF_E_INVALID_ARG;
            }
            if (a.type != cudaMemoryTypeHost) return HF_E_INVALID_ARG;  // pinned host memory only
        }
    }
    struct Piece {
        uint32_t cam, row0, rows;
    };
    std::vector<Piece> pieces;
    std::vector<uint32_t> first;  // chunk k is pieces[first[k], first[k + 1])
    {
        const uint64_t target = std::max((total_px + kStageChunks - 1) / kStageChunks, kMinChunkPx);
        uint64_t acc = 0;
        first.push_back(0);
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t w = cams[i].w, h = cams[i].h;
            for (uint32_t row = 0; row < h;) {
                const uint64_t want = (target - acc + w - 1) / w;  // rows that fill the chunk
                const uint32_t rows = (uint32_t)std::min<uint64_t>(h - row, want);
                pieces.push_back({i, row, rows});
                row += rows;
                acc += (uint64_t)rows * w;
                if (acc >= target) {
                    first.push_back((uint32_t)pieces.size());
                    acc = 0;
                }
            }
        }
        if (first.back() != pieces.size()) first.push_back((uint32_t)pieces.size());
    }
    auto piece_px = [&](const Piece &q) { return (size_t)cams[q.cam].w * q.rows; };
    // staging layout of a chunk: field by field, the chunk's pieces back to
    // back (so that pieces whose host buffers are adjacent need one copy)
    auto chunk_stage_bytes = [&](uint32_t k0, uint32_t k1) {
        size_t b = 0;
        for (int f = 0; f < 6; ++f) {
            size_t fb = 0;
            for (uint32_t k = k0; k < k1; ++k) fb += field_bytes(outs[pieces[k].cam], f) * piece_px(pieces[k]);
            b += (fb + kAlign - 1) & ~(kAlign - 1);
        }
        return b;
    };
    size_t need = 0;
    for (size_t k = 0; k + 1 < first.size(); ++k)
        need = std::max(need, chunk_stage_bytes(first[k], first[k + 1]));
    CK(cudaSetDevice(c->device));
    cudaStream_t s = o.cuda_stream ? (cudaStream_t)o.cuda_stream : c->stream;
    if (!c->copy_stream) {
        CK(cudaStreamCreateWithFlags(&c->render2, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->stage_start, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 4; ++b) {
            CK(cudaEventCreateWithFlags(&c->stage_ready[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->stage_free[b], cudaEventDisableTiming));
        }
    }
    if (need > c->hstage_half) {  // grow: nothing may still use the old buffers
        CK(cudaStreamSynchronize(c->render2));
        CK(cudaStreamSynchronize(c->copy_stream));
        for (int b = 0; b < 4; ++b) c->stage_busy[b] = false;
        sync_slots(c);
        if (c->d_hstage) cudaFree(c->d_hstage);
        c->d_hstage = nullptr;
        c->hstage_half = 0;
        const size_t half = (need + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
        if (cudaMalloc(&c->d_hstage, kBuffers * half) != cudaSuccess) {
            (void)cudaGetLastError();
            c->d_hstage = nullptr;
            return HF_E_OOM;
        }
        c->hstage_half = half;
    }
    hf_render_opts inner = o;
    inner.flags &= ~(HF_HOST_STAGED | HF_HOST_OUTPUTS | HF_SYNC);
    inner.cuda_stream = s;
    std::vector<hf_camera> band;
    std::vector<hf_outputs> dev;
    std::vector<const char *> srcs;  // staging of (piece, field), for the copies
    // the second render stream starts after the work already on the caller's
    const cudaStream_t rs[2] = {s, c->render2};
    CK(cudaEventRecord(c->stage_start, s));
    CK(cudaStreamWaitEvent(c->render2, c->stage_start, 0));
    for (size_t k = 0; k + 1 < first.size(); ++k) {
        const int b = (int)(k % kBuffers);
        const cudaStream_t ks = rs[k & 1];
        if (c->stage_busy[b]) CK(cudaStreamWaitEvent(ks, c->stage_free[b], 0));
        char *base = c->d_hstage + b * c->hstage_half;
        const uint32_t k0 = first[k], k1 = first[k + 1];
        band.assign(k1 - k0, hf_camera{});
        dev.assign(k1 - k0, hf_outputs{});
        srcs.assign((size_t)(k1 - k0) * 6, nullptr);
        for (uint32_t q = k0; q < k1; ++q) {
            const Piece &pc = pieces[q];
            hf_camera &bc = band[q - k0];
            bc = cams[pc.cam];
            const int64_t shift = (int64_t)bc.h - pc.rows - 2 * (int64_t)pc.row0;
            for (int i = 0; i < 3; ++i) bc.fwd[i] = (int32_t)(bc.fwd[i] + shift * bc.up[i]);
            bc.h = pc.rows;
        }
        size_t off = 0;
        for (int f = 0; f < 6; ++f) {
            for (uint32_t q = k0; q < k1; ++q) {
                const size_t fb = field_bytes(outs[pieces[q].cam], f) * piece_px(pieces[q]);
                if (!fb) continue;
                void *slot = base + off;
                off += fb;
                srcs[(size_t)(q - k0) * 6 + f] = static_cast<const char *>(slot);
                hf_outputs &d = dev[q - k0];
                switch (f) {
                    case 0: d.hit_cell = (uint32_t *)slot; break;
                    case 1: d.layer = (uint8_t *)slot; break;
                    case 2: d.face = (uint8_t *)slot; break;
                    case 3: d.depth = (float *)slot; break;
                    case 4: d.rgba = (uint32_t *)slot; break;
                    default: d.shadow = (uint8_t *)slot; break;
                }
            }
            off = (off + kAlign - 1) & ~(kAlign - 1);
        }
        inner.cuda_stream = ks;
        const int rc = hf_render(c, band.data(), k1 - k0, dev.data(), &inner);
        if (rc != HF_OK) return rc;
        CK(cudaEventRecord(c->stage_ready[b], ks));
        CK(cudaStreamWaitEvent(c->copy_stream, c->stage_ready[b], 0));
        // one copy per run of pieces whose host buffers of this field are
        // adjacent (their staging is adjacent by construction)
        for (int f = 0; f < 6; ++f) {
            char *run_dst = nullptr;
            const char *run_src = nullptr;
            size_t run_bytes = 0;
            for (uint32_t q = k0; q <= k1; ++q) {
                size_t fb = 0;
                char *dst = nullptr;
                const char *src = nullptr;
                if (q < k1) {
                    const Piece &pc = pieces[q];
                    const size_t eb = field_bytes(outs[pc.cam], f);
                    fb = eb * piece_px(pc);
                    if (fb) {
                        dst = static_cast<char *>(field_ptr(outs[pc.cam], f)) +
                              eb * cams[pc.cam].w * pc.row0;
                        src = srcs[(size_t)(q - k0) * 6 + f];
                    }
                }
                if (run_bytes && fb && dst == run_dst + run_bytes && src == run_src + run_bytes) {
                    run_bytes += fb;
                    continue;
                }
                if (run_bytes)
                    CK(cudaMemcpyAsync(run_dst, run_src, run_bytes, cudaMemcpyDeviceToHost,
                                       c->copy_stream));
                run_dst = dst;
                run_src = src;
                run_bytes = fb;
            }
        }
        CK(cudaEventRecord(c->stage_free[b], c->copy_stream));
        c->stage_busy[b] = true;
    }
    for (int b = 0; b < kBuffers; ++b)
        if (c->stage_busy[b]) CK(cudaStreamWaitEvent(s, c->stage_free[b], 0));
    if (o.flags & HF_SYNC) {
        CK(cudaStreamSynchronize(s));
        return read_status(c);
    }
    return HF_OK;
}

int hf_render(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
              const hf_render_opts *opts) {
    if (!c) return HF_E_INVALID_ARG;
    if (n == 0) return HF_OK;
    if (!cams || !outs || n > HF_MAX_CAMERAS) return HF_E_INVALID_ARG;
    hf_render_opts o{};
    if (opts) o = *opts;
    else o.mip_start = HF_MIP_AUTO;
    if (o.flags & HF_HOST_STAGED) {
        if (o.flags & (HF_HOST_OUTPUTS | HF_PLAIN | HF_NOWAIT)) return HF_E_INVALID_ARG;
        return render_host_staged(c, cams, n, outs, o);
    }
    const uint32_t tw = o.tile_w ? o.tile_w : 8, th = o.tile_h ? o.tile_h : 4;
    int32_t sun[3] = {o.sun[0], o.sun[1], o.sun[2]};
    if (sun[0] == 0 && sun[1] == 0 && sun[2] == 0)
        for (int i = 0; i < 3; ++i) sun[i] = kDefaultSun[i];
    for (int i = 0; i < 3; ++i)
        if (iabs64(sun[i]) >= kLimit21) return HF_E_INVALID_ARG;
    const bool shadows = (o.flags & HF_SHADOWS) != 0;
    const bool stats = (o.flags & HF_STATS) != 0;
    const uint32_t mip = o.mip_start == HF_MIP_AUTO ? hf::kDefaultMipStart : o.mip_start;
    const uint32_t mip_c = mip > c->L ? c->L : mip;
    const uint64_t guard = 4ull * (c->W + c->H) + 64;
    const uint32_t steps = o.max_steps ? o.max_steps : (uint32_t)(guard > 0x7FFFFFFF ? 0x7FFFFFFF : guard);
    if (steps > 0x7FFFFFFFu) return HF_E_INVALID_ARG;
    for (uint32_t i = 0; i < n; ++i)  // before anything is built or enqueued
        if (hf_validate_camera(c->W, c->H, &cams[i]) != HF_OK) return HF_E_INVALID_ARG;
    const uint32_t *bounds = nullptr;
    if (shadows) {
        const int brc = ensure_sun_bounds(c, sun, &bounds);
        if (brc != HF_OK) return brc;
    }
    Batch b;
    int rc = prepare_batch(c, cams, n, outs, tw, th, (o.flags & HF_NOWAIT) != 0, o.cuda_stream, b,
                           (o.flags & HF_HOST_OUTPUTS) != 0);
    if (rc != HF_OK) return rc;
    b.p.sun_bounds = bounds;
    Slot &s = c->slots[b.slot];
    hf::RenderParams &p = b.p;
    p.mip_start = (int32_t)mip_c;
    p.shadow_mip = (int32_t)(mip_c + hf::kShadowMipExtra > c->L ? c->L : mip_c + hf::kShadowMipExtra);
    p.max_steps = (int32_t)steps;
    const double sn = std::sqrt((double)sun[0] * sun[0] + (double)sun[1] * sun[1] +
                                (double)sun[2] * sun[2]);
    for (int i = 0; i < 3; ++i) {
        p.sun[i] = sun[i];
        p.sun_n[i] = (float)(sun[i] / sn);
    }
    // one camera: the plain launch (its grid covers the camera's tiles) spares
    // the persistent kernel's shared tile counter, which small tiles contend on
    if ((o.flags & HF_PLAIN) || (n == 1 && !(o.flags & HF_NOGRAPH))) {
        // each launch takes its camera record as a parameter: no copy to the device
        const auto *cd = (const hf::CamDev *)((const char *)s.h_staging + sizeof(hf::BatchHeader));
        for (uint32_t i = 0; i < n; ++i)
            if (hf::launch_trace_plain(p, shadows, stats, cd[i], b.tiles[i], b.stream))
                return HF_E_CUDA;
    } else if (o.flags & HF_NOGRAPH) {
        CK(cudaMemcpyAsync(s.d_scratch, s.h_staging, b.bytes, cudaMemcpyHostToDevice, b.stream));
        if (hf::launch_trace_batched(p, shadows, stats, c->sm_count * c->occ[shadows][stats],
                                     b.stream))
            return HF_E_CUDA;
    } else {
        GraphKey key{};
        key.bytes = (uint32_t)b.bucket;
        key.shadows = shadows;
        key.stats = stats;
        key.twl = (uint32_t)p.tile_w_log2;
        key.thl = (uint32_t)p.tile_h_log2;
        key.mip = mip_c;
        key.steps = steps;
        for (int i = 0; i < 3; ++i) key.sun[i] = sun[i];
        rc = launch_graph(c, s, key, p, shadows, stats, b.stream);
        if (rc != HF_OK) return rc;
    }
    return finish_batch(c, b, (o.flags & HF_SYNC) != 0);
}

int hf_render_march(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                    const hf_march_opts *opts) {
    if (!c) return HF_E_INVALID_ARG;
    if (n == 0) return HF_OK;
    if (!cams || !outs || n > HF_MAX_CAMERAS) return HF_E_INVALID_ARG;
    hf_march_opts o{};
    if (opts) o = *opts;
    hf::MarchParams m;
    m.steps = (int32_t)(o.steps ? o.steps : 128);
    m.bisections = (int32_t)(o.bisections ? o.bisections : 4);
    m.far_dist = o.far_dist != 0.0f ? o.far_dist : 600.0f;
    if (o.steps > 65536 || o.bisections > 65536 || !(m.far_dist > 0.0f)) return HF_E_INVALID_ARG;
    const uint32_t tw = o.tile_w ? o.tile_w : 8, th = o.tile_h ? o.tile_h : 4;
    if (c->occ_march < 1) return HF_E_CUDA;
    Batch b;
    int rc = prepare_batch(c, cams, n, outs, tw, th, false, o.cuda_stream, b);
    if (rc != HF_OK) return rc;
    Slot &s = c->slots[b.slot];
    CK(cudaMemcpyAsync(s.d_scratch, s.h_staging, b.bytes, cudaMemcpyHostToDevice, b.stream));
    if (hf::launch_march_batched(b.p, m, c->sm_count * c->occ_march, b.stream)) return HF_E_CUDA;
    return finish_batch(c, b, (o.flags & HF_SYNC) != 0);
}

int hf_scatter_footprint(const hf_camera *cam, float far_dist, hf_footprint *out) {
    if (!cam || !out || !(far_dist > 0.0f) || cam->w == 0 || cam->h == 0) return HF_E_INVALID_ARG;
    const double S = 65536.0;
    const double O[3] = {cam->origin[0] / S, cam->origin[1] / S, cam->origin[2] / S};
    const double rl = std::hypot((double)cam->right[0], (double)cam->right[1]);
    if (rl == 0.0) return HF_E_INVALID_ARG;
    const double rh[2] = {cam->right[0] / rl, cam->right[1] / rl}, fh[2] = {-rh[1], rh[0]};
    const double margin = 1.05;
    double ss[25], uu[25], rows[25];
    int np_ = 0;
    for (int ia = 0; ia < 5; ++ia)
        for (int ib = 0; ib < 5; ++ib) {  // a 5 x 5 grid of image points, edges included
            const double fa = -1.0 + 0.5 * ia, fb = -1.0 + 0.5 * ib;
            double d[3];
            for (int k = 0; k < 3; ++k)
                d[k] = cam->fwd[k] + fa * (cam->w - 1.0) * cam->right[k] + fb * (cam->h - 1.0) * cam->up[k];
            const double dl = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double t = far_dist / dl;
            if (d[2] < 0) t = std::min(t, O[2] / -d[2]);  // to the plane z = 0
            const double px = d[0] * t, py = d[1] * t;
            ss[np_] = px * fh[0] + py * fh[1];
            uu[np_] = std::fabs(px * rh[0] + py * rh[1]);
            rows[np_] = fb;
            ++np_;
        }
    double s_min = 0.0, s_max = -1e300, st = 0.0, sb = 0.0, ut = 0.0, ub = 0.0;
    for (int i = 0; i < np_; ++i) {
        s_min = std::min(s_min, ss[i]);
        s_max = std::max(s_max, ss[i]);
        if (rows[i] == 1.0) {  // top row of image points
            st += ss[i] / 5.0;
            ut = std::max(ut, uu[i]);
        } else if (rows[i] == -1.0) {  // bottom row
            sb += ss[i] / 5.0;
            ub = std::max(ub, uu[i]);
        }
    }
    const double ds = st - sb;
    const double k_lat = ds != 0.0 ? std::max(0.0, (ut - ub) / ds) : 0.0;
    double u0 = -1e300;
    for (int i = 0; i < np_; ++i) u0 = std::max(u0, uu[i] - k_lat * std::fabs(ss[i]));
    out->s_lo = (float)(s_min * margin - 1.0);
    out->s_hi = (float)std::max(1.0, s_max * margin + 1.0);
    out->k_lat = (float)(k_lat * margin);
    out->u_min = (float)(std::max(u0 * margin, 0.0) + 1.0);
    return HF_OK;
}

int hf_render_scatter(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_footprint *fps,
                      const hf_outputs *outs, const hf_scatter_opts *opts) {
    if (!c) return HF_E_INVALID_ARG;
    if (n == 0) return HF_OK;
    if (!cams || !outs || n > HF_MAX_CAMERAS) return HF_E_INVALID_ARG;
    hf_scatter_opts o{};
    if (opts) o = *opts;
    hf::ScatterParams sp{};
    sp.nu = o.nu ? o.nu : 1024;
    sp.nv = o.nv ? o.nv : 1024;
    sp.nz = o.nz ? o.nz : 16;
    sp.depth_max = o.depth_max != 0.0f ? o.depth_max : 1024.0f;
    sp.raw = (o.flags & HF_SCATTER_RAW) ? 1 : 0;
    if (sp.nu > 8192 || sp.nv > 8192 || sp.nz < 2 || sp.nz > 4096 || !(sp.depth_max > 0.0f))
        return HF_E_INVALID_ARG;
    int32_t sun[3] = {o.sun[0], o.sun[1], o.sun[2]};
    if (sun[0] == 0 && sun[1] == 0 && sun[2] == 0)
        for (int i = 0; i < 3; ++i) sun[i] = kDefaultSun[i];
    for (int i = 0; i < 3; ++i)
        if (iabs64(sun[i]) >= kLimit21) return HF_E_INVALID_ARG;
    // the resolved colour of each material: an up-facing surface lit by the sun
    static const float albedo[8][3] = HF_ALBEDO_TABLE;
    const double sl = std::sqrt((double)sun[0] * sun[0] + (double)sun[1] * sun[1] + (double)sun[2] * sun[2]);
    const double kl = hf::kAmbient + hf::kDiffuse * std::max(0.0, sun[2] / sl);
    for (int m = 0; m < 8; ++m) {
        uint32_t rgba = 0xFF000000u;
        for (int ch = 0; ch < 3; ++ch) {
            const double v = std::min(1.0, std::max(0.0, (double)albedo[m][ch] * kl));
            rgba |= (uint32_t)std::floor(255.0 * v + 0.5) << (8 * ch);
        }
        sp.colour[m] = rgba;
    }
    std::vector<hf_footprint> fp(n);
    uint32_t maxpix = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (!outs[i].hit_cell) return HF_E_INVALID_ARG;  // the screen buffer
        if (fps) {
            fp[i] = fps[i];
            if (!(fp[i].s_hi > fp[i].s_lo) || !(fp[i].k_lat >= 0.0f) || !(fp[i].u_min >= 0.0f))
                return HF_E_INVALID_ARG;
        } else if (hf_scatter_footprint(&cams[i], 600.0f, &fp[i]) != HF_OK) {
            return HF_E_INVALID_ARG;
        }
        if (cams[i].right[0] == 0 && cams[i].right[1] == 0) return HF_E_INVALID_ARG;
        maxpix = std::max(maxpix, cams[i].w * cams[i].h);
    }
    sp.max_pixels = maxpix;
    Batch b;
    int rc = prepare_batch(c, cams, n, outs, 8, 4, false, o.cuda_stream, b, false,
                           (size_t)n * sizeof(hf_footprint));
    if (rc != HF_OK) return rc;
    Slot &s = c->slots[b.slot];
    std::memcpy((char *)s.h_staging + sizeof(hf::BatchHeader) + (size_t)n * sizeof(hf::CamDev),
                fp.data(), (size_t)n * sizeof(hf_footprint));
    CK(cudaMemcpyAsync(s.d_scratch, s.h_staging, b.bytes, cudaMemcpyHostToDevice, b.stream));
    if (hf::launch_scatter(b.p, sp, n, b.stream)) return HF_E_CUDA;
    return finish_batch(c, b, (o.flags & HF_SYNC) != 0);
}

int hf_voxel_build(hf_ctx *c, const hf_voxel_desc *d) {
    if (!c || !d) return HF_E_INVALID_ARG;
    if (d->vx < 1 || d->vy < 1 || d->vz < 1 || d->vx > 64 || d->vy > 64 || d->vz > 256 ||
        d->levels > (uint32_t)hf::kVoxMaxLevels)
        return HF_E_INVALID_ARG;
    hf::VoxelDev v{};
    v.vx = (int32_t)d->vx;
    v.vy = (int32_t)d->vy;
    v.vz = (int32_t)d->vz;
    const int32_t n0[3] = {(int32_t)((c->W + d->vx - 1) / d->vx), (int32_t)((c->H + d->vy - 1) / d->vy),
                           (int32_t)((256 + d->vz - 1) / d->vz)};
    int32_t levels = (int32_t)d->levels;
    if (levels == 0) {  // enough levels that the top one is at most 8 voxels along every axis
        levels = 1;
        while (levels < hf::kVoxMaxLevels &&
               std::max({n0[0], n0[1], n0[2]}) > (8 << (levels - 1)))
            ++levels;
    }
    v.levels = levels;
    size_t off = 0;
    for (int l = 0; l < levels; ++l) {
        v.nx[l] = (n0[0] + (1 << l) - 1) >> l;
        v.ny[l] = (n0[1] + (1 << l) - 1) >> l;
        v.nz[l] = (n0[2] + (1 << l) - 1) >> l;
        v.tx[l] = (v.nx[l] + 7) >> 3;
        v.ty[l] = (v.ny[l] + 7) >> 3;
        v.off[l] = (uint32_t)off;
        off += (size_t)v.tx[l] * v.ty[l] * ((v.nz[l] + 7) >> 3) * 16;
    }
    CK(cudaSetDevice(c->device));
    for (auto &s : c->slots)
        if (s.pending) CK(cudaStreamWaitEvent(c->stream, s.done, 0));
    CK(cudaStreamSynchronize(c->stream));
    if (c->d_vox) {
        cudaFree(c->d_vox);
        c->d_vox = nullptr;
    }
    if (cudaMalloc(&c->d_vox, off * 4) != cudaSuccess) {
        (void)cudaGetLastError();
        c->d_vox = nullptr;
        return HF_E_OOM;
    }
    v.words = c->d_vox;
    c->vd = v;
    c->vox_words = off;
    CK(cudaMemsetAsync(c->d_vox, 0, off * 4, c->stream));
    if (hf::voxel_repair(c->wd, c->vd, 0, 0, (int32_t)c->W, (int32_t)c->H, true, c->stream))
        return HF_E_CUDA;
    CK(cudaEventRecord(c->edit_done, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HF_OK;
}

int hf_read_voxels(hf_ctx *c, uint32_t level, uint32_t *out, size_t *n_words) {
    if (!c || !n_words || !c->d_vox || level >= (uint32_t)c->vd.levels) return HF_E_INVALID_ARG;
    const size_t end = level + 1 < (uint32_t)c->vd.levels ? c->vd.off[level + 1] : c->vox_words;
    const size_t n = end - c->vd.off[level];
    if (!out) {
        *n_words = n;
        return HF_OK;
    }
    if (*n_words != n) return HF_E_INVALID_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(out, c->d_vox + c->vd.off[level], n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HF_OK;
}

int hf_render_voxel(hf_ctx *c, const hf_camera *cams, uint32_t n, const hf_outputs *outs,
                    const hf_voxel_opts *opts) {
    if (!c) return HF_E_INVALID_ARG;
    if (n == 0) return HF_OK;
    if (!cams || !outs || n > HF_MAX_CAMERAS || !c->d_vox) return HF_E_INVALID_ARG;
    hf_voxel_opts o{};
    if (opts) o = *opts;
    hf::VoxelParams q;
    q.outer = (int32_t)(o.outer ? o.outer : 1024);
    q.inner = (int32_t)(o.inner ? o.inner : 4);
    q.far_dist = o.far_dist != 0.0f ? o.far_dist : 600.0f;
    if (o.outer > 1u << 20 || o.inner > 4096 || !(q.far_dist > 0.0f)) return HF_E_INVALID_ARG;
    uint32_t maxpix = 0;
    for (uint32_t i = 0; i < n; ++i) maxpix = std::max(maxpix, cams[i].w * cams[i].h);
    Batch b;
    int rc = prepare_batch(c, cams, n, outs, 8, 4, false, o.cuda_stream, b);
    if (rc != HF_OK) return rc;
    Slot &s = c->slots[b.slot];
    CK(cudaMemcpyAsync(s.d_scratch, s.h_staging, b.bytes, cudaMemcpyHostToDevice, b.stream));
    if (hf::launch_voxel_trace(b.p, c->vd, q, n, maxpix, b.stream)) return HF_E_CUDA;
    return finish_batch(c, b, (o.flags & HF_SYNC) != 0);
}

}  // extern "C"
