// Many frames rendered into host memory with the device-to-host copies
// overlapped with rendering (jl_render_frames_to_host).
//
// Rendering a frame and copying its counts and colours to the host are both
// long for large frames (a 4096^2 frame is 100 MB of output).  Done one frame
// after the other, the copy time adds to the render time.  Here frame i is
// rendered on internal stream i mod D into device slot i mod D and copied out
// on the same stream, so up to D frames are in flight: copies of one frame
// run while the next frames render, and frames on different streams may also
// render side by side.  Stream order alone makes slot reuse safe (frame i + D
// is queued on the same stream after frame i's copies).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "jl_internal.h"

namespace jl {
int render_frame(Frame &F, int prec, const uint8_t *palette, cudaStream_t st, const Variant *vopt);
}

using namespace jl;

extern "C" int jl_render_frames_to_host(const jl_frame *frames, int32_t n, void *counts_host, uint8_t *rgba_host,
                                        float *hist_host, const uint8_t *palette, int32_t depth, void *stream)
{
    if (!frames || n < 1)
        return fail(JL_EINVAL, "frames must be non-NULL and n >= 1");
    if (depth == 0)
        depth = 6;
    if (depth < 1 || depth > 8)
        return fail(JL_EINVAL, "depth must be 0 (default 6) or 1..8");
    auto pad = [](size_t b) { return (b + 255) & ~(size_t)255; };

    struct Job {
        Frame F;
        int prec;
        size_t cbytes, rbytes, hbytes;
        const jl_frame *q;
    };
    std::vector<Job> jobs((size_t)n);
    size_t slot_bytes = 256;
    for (int i = 0; i < n; ++i) {
        const jl_frame &q = frames[i];
        const bool hc = q.counts_offset >= 0, hr = q.rgba_offset >= 0, hh = q.hist_offset >= 0;
        if ((hc && !counts_host) || (hr && !rgba_host) || (hh && !hist_host))
            return fail(JL_EINVAL, "frame " + std::to_string(i) + ": output offset given but base pointer is NULL");
        Job &j = jobs[(size_t)i];
        int rc = make_frame(q.cr, q.ci, q.rect, q.width, q.height, q.max_iter, q.precision, q.mode, q.count_type, hc,
                            hr, hh, &j.F, &j.prec);
        if (rc != JL_OK)
            return fail(rc, "frame " + std::to_string(i) + ": " + jl_last_error());
        const size_t npix = (size_t)q.width * (size_t)q.height;
        j.cbytes = hc ? npix * (q.count_type == JL_COUNT_U8 ? 1 : 2) : 0;
        j.rbytes = hr ? npix * 4 : 0;
        j.hbytes = hh ? ((size_t)q.max_iter + 1) * 4 : 0;
        j.q = &q;
        const size_t need = pad(j.cbytes) + pad(j.rbytes) + pad(j.hbytes);
        if (need > slot_bytes)
            slot_bytes = need;
    }
    if (depth > n)
        depth = n;

    cudaStream_t user = static_cast<cudaStream_t>(stream);
    std::vector<cudaStream_t> st((size_t)depth, nullptr);
    cudaEvent_t fork = nullptr;
    void *slots = nullptr;
    int rc = JL_OK;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    do {
        for (int s = 0; s < depth; ++s) {
            e = cudaStreamCreateWithFlags(&st[(size_t)s], cudaStreamNonBlocking);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamCreate"); break; }
        }
        if (rc != JL_OK)
            break;
        e = cudaMalloc(&slots, slot_bytes * (size_t)depth);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(frame slots)"); break; }
        // work already queued on the caller's stream comes first
        e = cudaEventRecord(fork, user);
        for (int s = 0; s < depth && e == cudaSuccess; ++s)
            e = cudaStreamWaitEvent(st[(size_t)s], fork, 0);
        if (e != cudaSuccess) { rc = cuda_fail(e, "stream fork"); break; }

        for (int i = 0; i < n && rc == JL_OK; ++i) {
            Job &j = jobs[(size_t)i];
            cudaStream_t s = st[(size_t)(i % depth)];
            uint8_t *b = static_cast<uint8_t *>(slots) + slot_bytes * (size_t)(i % depth);
            j.F.counts = j.cbytes ? b : nullptr;
            j.F.rgba = j.rbytes ? reinterpret_cast<uint32_t *>(b + pad(j.cbytes)) : nullptr;
            j.F.hist_bins = j.hbytes ? reinterpret_cast<uint32_t *>(b + pad(j.cbytes) + pad(j.rbytes)) : nullptr;
            rc = render_frame(j.F, j.prec, palette, s, nullptr);
            if (rc != JL_OK)
                break;
            if (j.cbytes) {
                e = cudaMemcpyAsync(static_cast<uint8_t *>(counts_host) + j.q->counts_offset, j.F.counts, j.cbytes,
                                    cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
            }
            if (j.rbytes) {
                e = cudaMemcpyAsync(rgba_host + j.q->rgba_offset, j.F.rgba, j.rbytes, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(rgba)"); break; }
            }
            if (j.hbytes) {
                e = cudaMemcpyAsync(reinterpret_cast<uint8_t *>(hist_host) + j.q->hist_offset, j.F.hist_bins,
                                    j.hbytes, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(hist)"); break; }
            }
        }
    } while (0);
    for (int s = 0; s < depth; ++s) {
        if (!st[(size_t)s])
            continue;
        cudaError_t e2 = cudaStreamSynchronize(st[(size_t)s]);
        if (rc == JL_OK && e2 != cudaSuccess)
            rc = cuda_fail(e2, "cudaStreamSynchronize");
        cudaStreamDestroy(st[(size_t)s]);
    }
    if (slots) {
        cudaError_t e2 = cudaFree(slots);
        if (rc == JL_OK && e2 != cudaSuccess)
            rc = cuda_fail(e2, "cudaFree(frame slots)");
    }
    cudaEventDestroy(fork);
    return rc;
}
