// hf_serve.cpp -- the native serving loop (hf_serve_replay): renders and edits
// over one resident world, with renders batched onto concurrent lanes and
// edits ordered between them (the paper's interactive setting, Section 4.4).
//
// The loop only schedules: every render goes through hf_render on a lane's
// stream and every edit through hf_edit, whose ordering rules (an edit waits
// for the renders already issued; a later render waits for the edit) give the
// version semantics.  Output memory comes from a stream-ordered pool the call
// owns; a batch's block is released when its completion event has fired.
//
// Clocks: arrivals and admissions are host times; completions are CUDA events.
// A reference event, then a few timed round trips (host time before an event
// is recorded on an idle stream, host time after it has fired) bracket the
// host time of the reference event; device times are mapped to the host clock
// through the middle of that bracket, so frame and edit-to-visible latencies
// subtract times on one clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

namespace {

constexpr uint32_t kMaxLanes = 64;

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    void *block = nullptr;
    uint64_t bytes = 0;
    std::vector<uint32_t> reqs;  // request indices of the batch in flight
};

uint64_t bytes_per_ray(uint32_t flags) {
    return 4 + 1 + 1 + 4 + 4 + ((flags & HF_SHADOWS) ? 1 : 0);  // cell, layer, face, depth, rgba
}

// Places one camera's output fields in a batch block (offset in bytes).
void carve(char *base, uint64_t &off, uint64_t px, bool shadows, hf_outputs &o) {
    auto take = [&](uint64_t sz) {
        void *p = base + off;
        off += (sz * px + 255) & ~uint64_t(255);
        return p;
    };
    o.hit_cell = static_cast<uint32_t *>(take(4));
    o.depth = static_cast<float *>(take(4));
    o.rgba = static_cast<uint32_t *>(take(4));
    o.layer = static_cast<uint8_t *>(take(1));
    o.face = static_cast<uint8_t *>(take(1));
    o.shadow = shadows ? static_cast<uint8_t *>(take(1)) : nullptr;
}

uint64_t batch_bytes(uint64_t px, bool shadows) {
    // per camera: each field rounded up to 256 bytes (carve's alignment)
    const uint64_t n = shadows ? 6 : 5;
    return px * bytes_per_ray(shadows ? HF_SHADOWS : 0) + n * 255;
}

bool own_outputs(const hf_outputs &o) {
    return o.hit_cell || o.layer || o.face || o.depth || o.rgba || o.shadow;
}

// pool bytes a render request takes (none when it brings its own buffers)
uint64_t pool_bytes(const hf_request &r, bool shadows) {
    return own_outputs(r.outs) ? 0 : batch_bytes((uint64_t)r.cam.w * r.cam.h, shadows);
}

}  // namespace

extern "C" int hf_serve_replay(hf_ctx *ctx, const hf_request *reqs, uint32_t n,
                               const hf_serve_opts *opts, hf_request_result *results) {
    if (!ctx || !opts || (n && (!reqs || !results))) return HF_E_INVALID_ARG;
    const hf_serve_opts o = *opts;
    if (o.lanes == 0 || o.lanes > kMaxLanes || o.max_batch == 0 || o.max_batch > HF_MAX_CAMERAS ||
        o.output_budget == 0 || (o.flags & ~HF_SHADOWS))
        return HF_E_INVALID_ARG;
    const bool shadows = (o.flags & HF_SHADOWS) != 0;
    for (uint32_t i = 0; i < n; ++i) {
        const hf_request &r = reqs[i];
        if (r.kind != HF_REQ_RENDER && r.kind != HF_REQ_EDIT) return HF_E_INVALID_ARG;
        if (i && r.arrival < reqs[i - 1].arrival) return HF_E_INVALID_ARG;
        if (r.kind == HF_REQ_RENDER && pool_bytes(r, shadows) > o.output_budget)
            return HF_E_INVALID_ARG;
    }
    if (n == 0) return HF_OK;
    hf_info_t info;
    int rc = hf_info(ctx, &info);
    if (rc != HF_OK) return rc;
    if (cudaSetDevice(info.device) != cudaSuccess) return HF_E_CUDA;

    // lanes and the output pool
    std::vector<Lane> lanes(o.lanes);
    cudaMemPool_t pool = nullptr;
    cudaEvent_t ref = nullptr;
    hf::CtxView view;
    if (hf::ctx_view(ctx, &view)) return HF_E_INVALID_ARG;
    // completion events of applied edits (recorded on the context's stream,
    // where hf_edit enqueues its copy and pyramid repair), created on demand
    std::vector<cudaEvent_t> edit_ev;
    std::vector<uint32_t> edit_req;
    size_t edit_retired = 0;
    auto cleanup = [&]() {
        for (cudaEvent_t e : edit_ev)
            if (e) cudaEventDestroy(e);
        for (auto &l : lanes) {
            if (l.stream) cudaStreamSynchronize(l.stream);
            if (l.block) cudaFreeAsync(l.block, l.stream);
            if (l.stream) cudaStreamSynchronize(l.stream);
            if (l.done) cudaEventDestroy(l.done);
            if (l.stream) cudaStreamDestroy(l.stream);
        }
        if (ref) cudaEventDestroy(ref);
        if (pool) cudaMemPoolDestroy(pool);
        (void)cudaGetLastError();
    };
    {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = info.device;
        bool ok = cudaMemPoolCreate(&pool, &props) == cudaSuccess;
        uint64_t keep = o.output_budget;  // keep freed blocks for reuse up to the budget
        ok = ok && cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
        ok = ok && cudaEventCreate(&ref) == cudaSuccess;
        for (auto &l : lanes) {
            ok = ok && cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaEventCreate(&l.done) == cudaSuccess;
        }
        if (!ok) {
            cleanup();
            return HF_E_CUDA;
        }
    }
    // device time 0: the reference event, taken once everything issued before
    // the replay (on the context's streams) has finished
    if (hf_sync(ctx) != HF_OK || cudaEventRecord(ref, lanes[0].stream) != cudaSuccess ||
        cudaEventSynchronize(ref) != cudaSuccess) {
        cleanup();
        return HF_E_CUDA;
    }
    using clock = std::chrono::steady_clock;
    const clock::time_point t0 = clock::now();
    auto now = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
    // host time of the reference event: each round trip gives
    // before <= dev + shift <= after for the event's device time dev
    double shift = 0.0;
    {
        cudaEvent_t cal = nullptr;
        double lo = -1e30, hi = 1e30, best = 1e30, best_mid = 0.0;
        bool ok = cudaEventCreate(&cal) == cudaSuccess;
        for (int k = 0; ok && k < 8; ++k) {
            const double before = now();
            ok = cudaEventRecord(cal, lanes[0].stream) == cudaSuccess &&
                 cudaEventSynchronize(cal) == cudaSuccess;
            const double after = now();
            float ms = 0.0f;
            ok = ok && cudaEventElapsedTime(&ms, ref, cal) == cudaSuccess;
            const double dev = ms / 1e3;
            lo = std::max(lo, before - dev);
            hi = std::min(hi, after - dev);
            if (after - before < best) {
                best = after - before;
                best_mid = 0.5 * (before + after) - dev;
            }
        }
        if (cal) cudaEventDestroy(cal);
        if (!ok) {
            cleanup();
            return HF_E_CUDA;
        }
        shift = lo <= hi ? 0.5 * (lo + hi) : best_mid;
    }

    hf_render_opts ro;
    std::memset(&ro, 0, sizeof(ro));
    ro.tile_w = o.tile_w;
    ro.tile_h = o.tile_h;
    ro.mip_start = o.mip_start;
    ro.flags = o.flags & HF_SHADOWS;

    std::deque<uint32_t> queue;
    uint32_t next = 0, version = 0, batches = 0;
    uint64_t mem_used = 0;
    int err = HF_OK;
    std::vector<hf_camera> cams;
    std::vector<hf_outputs> outs;

    auto retire = [&](Lane &l, bool block) -> bool {
        if (!l.busy) return false;
        if (block) {
            if (cudaEventSynchronize(l.done) != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
        } else {
            const cudaError_t q = cudaEventQuery(l.done);
            if (q == cudaErrorNotReady) return false;
            if (q != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ref, l.done) != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
        for (uint32_t i : l.reqs) results[i].done = ms / 1e3 + shift;
        if (l.block) cudaFreeAsync(l.block, l.stream);
        l.block = nullptr;
        mem_used -= l.bytes;
        l.bytes = 0;
        l.reqs.clear();
        l.busy = false;
        return true;
    };

    // edits complete in order on the context's stream
    auto retire_edits = [&](bool block) {
        while (edit_retired < edit_ev.size()) {
            cudaEvent_t e = edit_ev[edit_retired];
            if (block) {
                if (cudaEventSynchronize(e) != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
            } else {
                const cudaError_t q = cudaEventQuery(e);
                if (q == cudaErrorNotReady) return;
                if (q != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
            }
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ref, e) != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
            results[edit_req[edit_retired]].done = ms / 1e3 + shift;
            ++edit_retired;
        }
    };

    while (err == HF_OK && (next < n || !queue.empty())) {
        const double t = now();
        while (next < n && reqs[next].arrival <= t) queue.push_back(next++);
        for (auto &l : lanes) retire(l, false);
        retire_edits(false);
        // edits at the head of the queue, in order
        while (err == HF_OK && !queue.empty() && reqs[queue.front()].kind == HF_REQ_EDIT) {
            const uint32_t i = queue.front();
            queue.pop_front();
            const hf_request &r = reqs[i];
            results[i].admitted = now();
            const int e = hf_edit(ctx, r.x0, r.y0, r.w, r.h, r.cells, r.w);
            if (e != HF_OK) err = e;
            results[i].version = ++version;
            results[i].done = results[i].admitted;  // replaced when its event fires
            results[i].batch = 0xFFFFFFFFu;
            cudaEvent_t ev = nullptr;
            if (err == HF_OK && (cudaEventCreate(&ev) != cudaSuccess ||
                                 cudaEventRecord(ev, (cudaStream_t)view.stream) != cudaSuccess))
                err = HF_E_CUDA;
            if (ev) {
                edit_ev.push_back(ev);
                edit_req.push_back(i);
            }
        }
        // one batch of renders on a free lane
        Lane *free_lane = nullptr;
        for (auto &l : lanes)
            if (!l.busy) {
                free_lane = &l;
                break;
            }
        if (err == HF_OK && free_lane && !queue.empty()) {
            cams.clear();
            std::vector<uint32_t> idx;
            uint64_t bytes = 0;
            while (!queue.empty() && idx.size() < o.max_batch &&
                   reqs[queue.front()].kind == HF_REQ_RENDER) {
                const hf_request &r = reqs[queue.front()];
                const uint64_t b = pool_bytes(r, shadows);
                if (mem_used + bytes + b > o.output_budget) break;
                bytes += b;
                idx.push_back(queue.front());
                cams.push_back(r.cam);
                queue.pop_front();
            }
            if (!idx.empty()) {
                Lane &l = *free_lane;
                void *block = nullptr;
                if (bytes && cudaMallocFromPoolAsync(&block, bytes, pool, l.stream) != cudaSuccess) {
                    err = HF_E_OOM;
                    break;
                }
                outs.assign(idx.size(), hf_outputs{});
                uint64_t off = 0;
                for (size_t k = 0; k < idx.size(); ++k) {
                    if (own_outputs(reqs[idx[k]].outs))
                        outs[k] = reqs[idx[k]].outs;
                    else
                        carve(static_cast<char *>(block), off, (uint64_t)cams[k].w * cams[k].h,
                              shadows, outs[k]);
                }
                const double ta = now();
                for (uint32_t i : idx) {
                    results[i].admitted = ta;
                    results[i].version = version;
                    results[i].batch = batches;
                }
                ro.cuda_stream = l.stream;
                const int e = hf_render(ctx, cams.data(), (uint32_t)cams.size(), outs.data(), &ro);
                l.block = block;
                l.bytes = bytes;
                l.reqs = idx;
                l.busy = true;
                mem_used += bytes;
                ++batches;
                if (e != HF_OK) err = e;
                if (cudaEventRecord(l.done, l.stream) != cudaSuccess && err == HF_OK) err = HF_E_CUDA;
                continue;
            }
        }
        // nothing to admit now: wait for an arrival or a completion
        if (queue.empty() || !free_lane) std::this_thread::yield();
    }
    for (auto &l : lanes) retire(l, true);
    retire_edits(true);
    const int sync = hf_sync(ctx);
    cleanup();
    if (err != HF_OK) return err;
    return sync;
}
