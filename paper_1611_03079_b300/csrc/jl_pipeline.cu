// Many frames rendered into host memory with the device-to-host copies
// overlapped with rendering (jl_host_plan_*, jl_render_frames_to_host).
//
// Rendering a frame and copying its counts and colours to the host are both
// long for large frames (a 4096^2 frame is 100 MB of output).  Done one frame
// after the other, the copy time adds to the render time.  Here frame i is
// rendered on internal stream i mod D into device slot i mod D and copied out
// on the same stream, so up to D frames are in flight: copies of one frame
// run while the next frames render, and frames on different streams may also
// render side by side.  Stream order alone makes slot reuse safe (frame i + D
// is queued on the same stream after frame i's copies).
//
// A plan does the once-per-frame-set work at creation: validation, the
// coordinate tables of every frame, the device slots and the streams.  A run
// then only launches the escape kernels and the copies.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "jl_internal.h"

namespace jl {
int launch_frame(Frame &F, int prec, const uint8_t *palette, void *ctl, cudaStream_t st, const Variant *vopt);
}

using namespace jl;

struct jl_host_plan {
    int device = 0;
    int n = 0, depth = 0;
    std::vector<Frame> F;
    std::vector<int> prec;
    std::vector<size_t> cbytes, rbytes, hbytes, ctl_off;
    std::vector<int64_t> coff, roff, hoff;
    void *counts_host = nullptr;
    uint8_t *rgba_host = nullptr;
    float *hist_host = nullptr;
    uint8_t palette[1024];
    bool has_palette = false;
    std::vector<cudaStream_t> st;
    cudaEvent_t fork = nullptr;
    void *slots = nullptr;
    size_t slot_bytes = 0;
    void *tables = nullptr;  // coordinate tables and a 256-byte control block per frame
};

static size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

static void destroy_host_plan(jl_host_plan *p)
{
    if (!p)
        return;
    for (cudaStream_t s : p->st)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (p->fork)
        cudaEventDestroy(p->fork);
    cudaFree(p->slots);
    cudaFree(p->tables);
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
    if (depth == 0)
        depth = 6;
    if (depth < 1 || depth > 8)
        return fail(JL_EINVAL, "depth must be 0 (default 6) or 1..8");
    jl_host_plan *p = new jl_host_plan();
    p->n = n;
    p->depth = depth > n ? n : depth;
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
        p->ctl_off[(size_t)i] = table_bytes;
        table_bytes += 256;
    }
    p->slot_bytes = slot_bytes;
    int rc = JL_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    do {
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); break; }
        p->st.assign((size_t)p->depth, nullptr);
        for (int s = 0; s < p->depth; ++s) {
            e = cudaStreamCreateWithFlags(&p->st[(size_t)s], cudaStreamNonBlocking);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamCreate"); break; }
        }
        if (rc != JL_OK)
            break;
        e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventCreate"); break; }
        e = cudaMalloc(&p->slots, slot_bytes * (size_t)p->depth);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(frame slots)"); break; }
        e = cudaMalloc(&p->tables, table_bytes);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(coordinate tables)"); break; }
        // coordinate tables of every frame, once
        for (int i = 0; i < n && rc == JL_OK; ++i) {
            Frame &F = p->F[(size_t)i];
            const size_t esz = p->prec[(size_t)i] == JL_FP64 ? 8 : 4;
            uint8_t *base = static_cast<uint8_t *>(p->tables) + table_off[(size_t)i];
            F.xs = base;
            F.ys = base + (size_t)F.W * esz;
            e = launch_coords(nullptr, &F, 1, p->st[0]);
            if (e != cudaSuccess)
                rc = cuda_fail(e, "coords kernel launch");
        }
        if (rc != JL_OK)
            break;
        e = cudaStreamSynchronize(p->st[0]);
        if (e != cudaSuccess) { rc = cuda_fail(e, "coordinate tables"); break; }
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
    for (int s = 0; s < p->depth && e == cudaSuccess; ++s)
        e = cudaStreamWaitEvent(p->st[(size_t)s], p->fork, 0);
    if (e != cudaSuccess)
        rc = cuda_fail(e, "stream fork");
    const uint8_t *pal = p->has_palette ? p->palette : nullptr;
    for (int i = 0; i < p->n && rc == JL_OK; ++i) {
        const size_t k = (size_t)i;
        Frame F = p->F[k];
        cudaStream_t s = p->st[(size_t)(i % p->depth)];
        uint8_t *b = static_cast<uint8_t *>(p->slots) + p->slot_bytes * (size_t)(i % p->depth);
        F.counts = p->cbytes[k] ? b : nullptr;
        F.rgba = p->rbytes[k] ? reinterpret_cast<uint32_t *>(b + pad256(p->cbytes[k])) : nullptr;
        F.hist_bins = p->hbytes[k] ? reinterpret_cast<uint32_t *>(b + pad256(p->cbytes[k]) + pad256(p->rbytes[k]))
                                   : nullptr;
        rc = launch_frame(F, p->prec[k], pal, static_cast<uint8_t *>(p->tables) + p->ctl_off[k], s, nullptr);
        if (rc != JL_OK)
            break;
        if (p->cbytes[k]) {
            e = cudaMemcpyAsync(static_cast<uint8_t *>(p->counts_host) + p->coff[k], F.counts, p->cbytes[k],
                                cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
        }
        if (p->rbytes[k]) {
            e = cudaMemcpyAsync(p->rgba_host + p->roff[k], F.rgba, p->rbytes[k], cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(rgba)"); break; }
        }
        if (p->hbytes[k]) {
            e = cudaMemcpyAsync(reinterpret_cast<uint8_t *>(p->hist_host) + p->hoff[k], F.hist_bins, p->hbytes[k],
                                cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(hist)"); break; }
        }
    }
    for (int s = 0; s < p->depth; ++s) {
        cudaError_t e2 = cudaStreamSynchronize(p->st[(size_t)s]);
        if (rc == JL_OK && e2 != cudaSuccess)
            rc = cuda_fail(e2, "cudaStreamSynchronize");
    }
    return rc;
}

void jl_host_plan_destroy(jl_host_plan *p) { destroy_host_plan(p); }

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
