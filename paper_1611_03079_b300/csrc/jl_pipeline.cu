// Many frames rendered into host memory with the device-to-host copies
// overlapped with rendering (jl_host_plan_*, jl_render_frames_to_host).
//
// Rendering a frame and copying its counts and colours to the host are both
// long for large frames (a 4096^2 frame is 96 MB of output, 1.7 ms over a
// 57 GB/s link).  Done one frame after the other, the copy time adds to the
// render time.  Here the renders and the copies run on separate internal
// streams: frame i renders on render stream i mod R into device slot
// i mod S and is copied out on copy stream i mod C once an event says its
// render is done.  A render never waits for a copy except to reuse a slot
// (frame i + S waits for frame i's copy), so with as many slots as frames
// the renders follow one another as closely as a single batched launch while
// the copy engine drains finished frames behind them; only the last frame's
// copy is left outside the rendering.  Several render streams let the next
// frame's blocks fill the SMs that the tail of the previous frame leaves idle.
// The last frame is rendered as row bands (launches over row ranges of the
// frame, sharing its coordinate tables, so every pixel gets the coordinates
// of the whole frame) spread over the render streams, each band copied out
// when it is done: what remains outside the rendering is the last band's copy.
//
// A plan does the once-per-frame-set work at creation: validation, the
// coordinate tables of every frame, the device slots, streams and events.  A
// run then only launches the escape kernels and the copies.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "jl_internal.h"


using namespace jl;

// One launch of the plan: rows [row0, row0 + rows) of frame `frame`, with
// its own control block (work counter and status word) at ctl_off.
struct Unit {
    int frame, row0, rows;
    size_t ctl_off;
};

struct jl_host_plan {
    int device = 0;
    int n = 0, depth = 0;  // depth = device slots (frames whose outputs may be on the device at once)
    std::vector<Frame> F;
    std::vector<int> prec;
    std::vector<size_t> cbytes, rbytes, hbytes, ctl_off;
    std::vector<int64_t> coff, roff, hoff;
    void *counts_host = nullptr;
    uint8_t *rgba_host = nullptr;
    float *hist_host = nullptr;
    uint8_t palette[1024];
    bool has_palette = false;
    std::vector<Unit> units;                  // launches in order: whole frames, then the last frame's bands
    std::vector<cudaStream_t> rs, cs;         // render streams, copy streams
    std::vector<cudaEvent_t> rendered;        // per unit: its render is done
    std::vector<cudaEvent_t> copied;          // per slot: the last copy out of it
    cudaEvent_t fork = nullptr;
    cudaEvent_t tables_ready = nullptr;       // the banded frame's coordinate tables are written
    void *slots = nullptr;
    size_t slot_bytes = 0;
    void *tables = nullptr;  // coordinate tables, a 256-byte control block per frame and per extra band
    // binary64 units: the certified passes' two lists of each render stream
    // (units on one stream run one after the other), list_cap entries each
    uint64_t *lists = nullptr;
    int64_t list_cap = 0;
};

static size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

// At most this many render and copy streams.  Together they stay within the
// device's default 8 hardware work queues, so no stream shares a queue (and a
// false dependency) with another.  Four render streams were the fastest of
// 2, 3, 4 and 6 on the 16-frame 4096^2 sweep (each fills the tail of one
// launch with the next).
static constexpr int kRenderStreams = 4, kCopyStreams = 2;
// The last frame is split into row bands when its outputs (counts + RGBA,
// no histogram) reach kBandMinBytes: bands of about kBandBytes, at most
// kMaxBands, each a multiple of 32 rows (whole 32 x 32 tiles).  Four bands
// beat one and eight on the sweep: more bands add launch tails.
static constexpr size_t kBandMinBytes = (size_t)8 << 20, kBandBytes = (size_t)8 << 20;
static constexpr int kMaxBands = 4;
// Default slot count: one per frame up to 16, and at most 4 GiB of slots.
static constexpr int kDefaultSlots = 16;
static constexpr size_t kDefaultSlotBudget = (size_t)4 << 30;

static void destroy_host_plan(jl_host_plan *p)
{
    if (!p)
        return;
    for (auto *v : {&p->rs, &p->cs})
        for (cudaStream_t s : *v)
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
    for (auto *v : {&p->rendered, &p->copied})
        for (cudaEvent_t e : *v)
            if (e)
                cudaEventDestroy(e);
    if (p->fork)
        cudaEventDestroy(p->fork);
    if (p->tables_ready)
        cudaEventDestroy(p->tables_ready);
    cudaFree(p->slots);
    cudaFree(p->tables);
    cudaFree(p->lists);
    delete p;
}

extern "C" {

int jl_host_plan_create(const jl_frame *frames, int32_t n, void *counts_host, uint8_t *rgba_host, float *hist_host,
                        const uint8_t *palette, int32_t depth, jl_host_plan **out)
{
    if (!out)
        return fail(JL_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (!frames || n < 1)
        return fail(JL_EINVAL, "frames must be non-NULL and n >= 1");
    if (depth < 0 || depth > 64)
        return fail(JL_EINVAL, "depth must be 0 (default) or 1..64");
    jl_host_plan *p = new jl_host_plan();
    p->n = n;
    p->counts_host = counts_host;
    p->rgba_host = rgba_host;
    p->hist_host = hist_host;
    if (palette) {
        memcpy(p->palette, palette, 1024);
        p->has_palette = true;
    }
    p->F.resize((size_t)n);
    p->prec.resize((size_t)n);
    p->cbytes.resize((size_t)n);
    p->rbytes.resize((size_t)n);
    p->hbytes.resize((size_t)n);
    p->ctl_off.resize((size_t)n);
    p->coff.resize((size_t)n);
    p->roff.resize((size_t)n);
    p->hoff.resize((size_t)n);
    size_t slot_bytes = 256, table_bytes = 0;
    std::vector<size_t> table_off((size_t)n);
    for (int i = 0; i < n; ++i) {
        const jl_frame &q = frames[i];
        const bool hc = q.counts_offset >= 0, hr = q.rgba_offset >= 0, hh = q.hist_offset >= 0;
        if ((hc && !counts_host) || (hr && !rgba_host) || (hh && !hist_host)) {
            destroy_host_plan(p);
            return fail(JL_EINVAL, "frame " + std::to_string(i) + ": output offset given but base pointer is NULL");
        }
        int rc = make_frame(q.cr, q.ci, q.rect, q.width, q.height, q.max_iter, q.precision, q.mode, q.count_type, hc,
                            hr, hh, &p->F[(size_t)i], &p->prec[(size_t)i]);
        if (rc != JL_OK) {
            const std::string msg = jl_last_error();
            destroy_host_plan(p);
            return fail(rc, "frame " + std::to_string(i) + ": " + msg);
        }
        const size_t npix = (size_t)q.width * (size_t)q.height;
        p->cbytes[(size_t)i] = hc ? npix * (q.count_type == JL_COUNT_U8 ? 1 : 2) : 0;
        p->rbytes[(size_t)i] = hr ? npix * 4 : 0;
        p->hbytes[(size_t)i] = hh ? ((size_t)q.max_iter + 1) * 4 : 0;
        p->coff[(size_t)i] = q.counts_offset;
        p->roff[(size_t)i] = q.rgba_offset;
        p->hoff[(size_t)i] = q.hist_offset;
        const size_t need = pad256(p->cbytes[(size_t)i]) + pad256(p->rbytes[(size_t)i]) + pad256(p->hbytes[(size_t)i]);
        if (need > slot_bytes)
            slot_bytes = need;
        const size_t esz = p->prec[(size_t)i] == JL_FP64 ? 8 : 4;
        table_off[(size_t)i] = table_bytes;
        table_bytes += pad256(((size_t)q.width + (size_t)q.height) * esz);
        if (p->prec[(size_t)i] == JL_FP64)  // binary32 roundings and remainders for the certified passes
            table_bytes += pad256(((size_t)q.width + (size_t)q.height) * 8);
        p->ctl_off[(size_t)i] = table_bytes;
        table_bytes += 256;
    }
    // launches: every frame whole, the last one in row bands (see kBandBytes)
    for (int i = 0; i < n; ++i)
        if (i < n - 1 || p->hbytes[(size_t)i] || p->cbytes[(size_t)i] + p->rbytes[(size_t)i] < kBandMinBytes) {
            p->units.push_back(Unit{i, 0, p->F[(size_t)i].H, p->ctl_off[(size_t)i]});
        } else {
            const Frame &F = p->F[(size_t)i];
            const size_t bytes = p->cbytes[(size_t)i] + p->rbytes[(size_t)i];
            int bands = (int)((bytes + kBandBytes - 1) / kBandBytes);
            bands = bands > kMaxBands ? kMaxBands : bands;
            int rows = (F.H + bands - 1) / bands;
            rows = (rows + 31) & ~31;
            for (int r0 = 0; r0 < F.H; r0 += rows) {
                const size_t ctl = r0 == 0 ? p->ctl_off[(size_t)i] : table_bytes;
                if (r0 > 0)
                    table_bytes += 256;
                p->units.push_back(Unit{i, r0, F.H - r0 < rows ? F.H - r0 : rows, ctl});
            }
        }
    p->slot_bytes = slot_bytes;
    const int nr = n < kRenderStreams ? n : kRenderStreams, nc = n < kCopyStreams ? n : kCopyStreams;
    for (size_t u = 0; u < p->units.size(); ++u) {
        const Unit &U = p->units[u];
        if (p->prec[(size_t)U.frame] == JL_FP64) {
            const int64_t px = (int64_t)U.rows * p->F[(size_t)U.frame].W;
            p->list_cap = px > p->list_cap ? px : p->list_cap;
        }
    }
    if (depth == 0) {
        size_t fit = kDefaultSlotBudget / slot_bytes;
        depth = (int)(fit < (size_t)kDefaultSlots ? (fit < 1 ? 1 : fit) : kDefaultSlots);
    }
    p->depth = depth > n ? n : depth;
    int rc = JL_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    do {
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); break; }
        p->rs.assign((size_t)nr, nullptr);
        p->cs.assign((size_t)nc, nullptr);
        for (auto *v : {&p->rs, &p->cs})
            for (cudaStream_t &s : *v)
                if (rc == JL_OK && (e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
                    rc = cuda_fail(e, "cudaStreamCreate");
        p->rendered.assign(p->units.size(), nullptr);
        p->copied.assign((size_t)p->depth, nullptr);
        for (auto *v : {&p->rendered, &p->copied})
            for (cudaEvent_t &ev : *v)
                if (rc == JL_OK && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                    rc = cuda_fail(e, "cudaEventCreate");
        if (rc != JL_OK)
            break;
        e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventCreate"); break; }
        e = cudaMalloc(&p->slots, slot_bytes * (size_t)p->depth);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(frame slots)"); break; }
        e = cudaMalloc(&p->tables, table_bytes);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(coordinate tables)"); break; }
        if (p->list_cap > 0) {
            e = cudaMalloc(&p->lists, (size_t)p->list_cap * sizeof(uint64_t) * 2 * (size_t)nr);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(certified pass lists)"); break; }
        }
        // where each frame's coordinate tables live (jl_host_plan_run fills them)
        for (int i = 0; i < n; ++i) {
            Frame &F = p->F[(size_t)i];
            const size_t esz = p->prec[(size_t)i] == JL_FP64 ? 8 : 4;
            uint8_t *base = static_cast<uint8_t *>(p->tables) + table_off[(size_t)i];
            F.xs = base;
            F.ys = base + (size_t)F.W * esz;
            if (esz == 8) {
                F.xs32 = reinterpret_cast<const float *>(base + pad256(((size_t)F.W + (size_t)F.H) * 8));
                F.ys32 = F.xs32 + F.W;
                F.xs32lo = F.ys32 + F.H;
                F.ys32lo = F.xs32lo + F.W;
            }
        }
        e = cudaEventCreateWithFlags(&p->tables_ready, cudaEventDisableTiming);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventCreate"); break; }
    } while (0);
    if (rc != JL_OK) {
        destroy_host_plan(p);
        return rc;
    }
    *out = p;
    return JL_OK;
}

int jl_host_plan_run(jl_host_plan *p, void *stream)
{
    if (!p)
        return fail(JL_EINVAL, "plan must not be NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return fail(JL_EINVAL, "the plan belongs to another device");
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    int rc = JL_OK;
    // work already queued on the caller's stream comes first
    cudaError_t e = cudaEventRecord(p->fork, user);
    for (auto *v : {&p->rs, &p->cs})
        for (cudaStream_t s : *v)
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(s, p->fork, 0);
    if (e != cudaSuccess)
        rc = cuda_fail(e, "stream fork");
    const uint8_t *pal = p->has_palette ? p->palette : nullptr;
    const size_t nr = p->rs.size(), nc = p->cs.size();
    for (size_t u0 = 0; u0 < p->units.size() && rc == JL_OK;) {
        // the units of one frame: [u0, u1)
        const size_t k = (size_t)p->units[u0].frame, slot = k % (size_t)p->depth;
        size_t u1 = u0 + 1;
        while (u1 < p->units.size() && (size_t)p->units[u1].frame == k)
            ++u1;
        const Frame &F0 = p->F[k];
        const size_t csz = F0.count_type == JL_COUNT_U8 ? 1 : 2, esz = p->prec[k] == JL_FP64 ? 8 : 4;
        uint8_t *b = static_cast<uint8_t *>(p->slots) + p->slot_bytes * slot;
        uint8_t *cnt = p->cbytes[k] ? b : nullptr;
        uint32_t *rgba = p->rbytes[k] ? reinterpret_cast<uint32_t *>(b + pad256(p->cbytes[k])) : nullptr;
        uint32_t *bins = p->hbytes[k] ? reinterpret_cast<uint32_t *>(b + pad256(p->cbytes[k]) + pad256(p->rbytes[k]))
                                      : nullptr;
        cudaStream_t c = p->cs[k % nc];
        // step A1 of every run: the frame's coordinate tables from its
        // descriptor (which reaches the device as the kernel's parameters),
        // on the stream of its first unit; units on other streams (row bands)
        // wait for them
        e = launch_coords(nullptr, &F0, 1, p->rs[u0 % nr]);
        if (e == cudaSuccess && u1 - u0 > 1)
            e = cudaEventRecord(p->tables_ready, p->rs[u0 % nr]);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "coords kernel launch");
            break;
        }
        for (size_t u = u0; u < u1 && rc == JL_OK; ++u) {
            const Unit &U = p->units[u];
            cudaStream_t r = p->rs[u % nr];
            if (u > u0 && (u % nr) != (u0 % nr) && (e = cudaStreamWaitEvent(r, p->tables_ready, 0)) != cudaSuccess) {
                rc = cuda_fail(e, "cudaStreamWaitEvent(tables ready)");
                break;
            }
            // the slot's previous frame (k - depth) must be copied out first
            if (k >= (size_t)p->depth && (e = cudaStreamWaitEvent(r, p->copied[slot], 0)) != cudaSuccess) {
                rc = cuda_fail(e, "cudaStreamWaitEvent(slot copied)");
                break;
            }
            Frame F = F0;
            const size_t pix0 = (size_t)U.row0 * (size_t)F0.W;
            F.counts = cnt ? cnt + pix0 * csz : nullptr;
            F.rgba = rgba ? rgba + pix0 : nullptr;
            F.hist_bins = bins;  // only whole frames carry a histogram
            if (U.rows != F0.H) {
                F.H = U.rows;
                F.ys = static_cast<const uint8_t *>(F0.ys) + (size_t)U.row0 * esz;
                if (F0.ys32) {
                    F.ys32 = F0.ys32 + U.row0;
                    F.ys32lo = F0.ys32lo + U.row0;
                }
                F.chunk_count = F0.rows_per_chunk > 1 ? (U.rows + F0.rows_per_chunk - 1) / F0.rows_per_chunk
                                                      : U.rows * F0.chunks_per_row;
                F.tile_count = F0.tiles_x * ((U.rows + 31) / 32);
            }
            uint64_t *list = p->lists ? p->lists + (size_t)p->list_cap * 2 * (u % nr) : nullptr;
            rc = launch_frame(F, p->prec[k], pal, static_cast<uint8_t *>(p->tables) + U.ctl_off, r, nullptr, list,
                              p->list_cap, list ? list + p->list_cap : nullptr);
            if (rc != JL_OK)
                break;
            if ((e = cudaEventRecord(p->rendered[u], r)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(c, p->rendered[u], 0)) != cudaSuccess) {
                rc = cuda_fail(e, "render -> copy event");
                break;
            }
            const size_t npx = (size_t)U.rows * (size_t)F0.W;
            if (cnt) {
                e = cudaMemcpyAsync(static_cast<uint8_t *>(p->counts_host) + p->coff[k] + pix0 * csz, F.counts,
                                    npx * csz, cudaMemcpyDeviceToHost, c);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
            }
            if (rgba) {
                e = cudaMemcpyAsync(p->rgba_host + p->roff[k] + pix0 * 4, F.rgba, npx * 4, cudaMemcpyDeviceToHost, c);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(rgba)"); break; }
            }
            if (bins) {
                e = cudaMemcpyAsync(reinterpret_cast<uint8_t *>(p->hist_host) + p->hoff[k], bins, p->hbytes[k],
                                    cudaMemcpyDeviceToHost, c);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(hist)"); break; }
            }
        }
        if (rc == JL_OK && (e = cudaEventRecord(p->copied[slot], c)) != cudaSuccess)
            rc = cuda_fail(e, "cudaEventRecord(slot copied)");
        u0 = u1;
    }
    // every stream is drained before returning, also after an error, so that
    // no copy into the caller's buffers is still running when the call returns
    for (auto *v : {&p->rs, &p->cs})
        for (cudaStream_t s : *v) {
            cudaError_t e2 = cudaStreamSynchronize(s);
            if (rc == JL_OK && e2 != cudaSuccess)
                rc = cuda_fail(e2, "cudaStreamSynchronize");
        }
    return rc;
}

void jl_host_plan_destroy(jl_host_plan *p) { destroy_host_plan(p); }

int32_t jl_host_plan_launches(const jl_host_plan *p) { return p ? (int32_t)p->units.size() : -1; }

int jl_render_frames_to_host(const jl_frame *frames, int32_t n, void *counts_host, uint8_t *rgba_host,
                             float *hist_host, const uint8_t *palette, int32_t depth, void *stream)
{
    jl_host_plan *p = nullptr;
    int rc = jl_host_plan_create(frames, n, counts_host, rgba_host, hist_host, palette, depth, &p);
    if (rc != JL_OK)
        return rc;
    rc = jl_host_plan_run(p, stream);
    destroy_host_plan(p);
    return rc;
}

}  // extern "C"
