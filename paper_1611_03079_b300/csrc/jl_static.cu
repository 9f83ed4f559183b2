// jl_render_static: a single-frame render that allocates nothing.
//
// Some callers cannot allocate device memory when they render: a real-time
// display loop that must not stall on an allocation (cudaMalloc can
// synchronise the whole device), or a process whose device memory is reserved
// up front by another allocator (for example a framework's caching
// allocator), where any further allocation fails or fragments that
// reservation.  This entry point serves them: its scratch (the per-frame
// coordinate tables, the work counter and the status word) lives in the
// file-scope array below instead of stream-ordered allocations.  Every GPU
// that loads this library holds the array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "jl_internal.h"

namespace jl {

static __device__ __align__(256) uint8_t g_static_scratch[JL_STATIC_SCRATCH_BYTES];

// In host code `g_static_scratch` names a host-side stand-in, not device
// memory, so the kernels get the device address looked up here: once per
// device, with that device current.
static constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void *g_static_addr[kMaxDevices] = {};

static int static_scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(JL_EUNSUPPORTED, "device index beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return JL_OK;
}

}  // namespace jl

using namespace jl;

extern "C" int jl_render_static(double cr, double ci, jl_rect rect, int32_t width, int32_t height,
                                int32_t max_iter, int32_t precision, int32_t mode, int32_t count_type,
                                void *counts, uint8_t *rgba, const uint8_t *palette, float *hist, void *stream)
{
    Frame F;
    int prec = 0;
    int rc = make_frame(cr, ci, rect, width, height, max_iter, precision, mode, count_type, counts != nullptr,
                        rgba != nullptr, hist != nullptr, &F, &prec);
    if (rc != JL_OK)
        return rc;
    const size_t esz = prec == JL_FP64 ? 8 : 4;
    const size_t coord_bytes = ((size_t)F.W + (size_t)F.H) * esz;
    const size_t coord_pad = (coord_bytes + 255) & ~(size_t)255;
    if (coord_pad + 256 > (size_t)JL_STATIC_SCRATCH_BYTES)
        return fail(JL_EINVAL, "jl_render_static: (width + height) * " + std::to_string(esz) +
                                   " bytes of coordinate tables exceed the static scratch of " +
                                   std::to_string((size_t)JL_STATIC_SCRATCH_BYTES) +
                                   " bytes (limit: width + height <= " +
                                   std::to_string(((size_t)JL_STATIC_SCRATCH_BYTES - 256) / esz) + ")");
    void *scratch = nullptr;
    rc = static_scratch_address(&scratch);
    if (rc != JL_OK)
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(scratch);
    F.xs = base;
    F.ys = base + (size_t)F.W * esz;
    F.counts = static_cast<uint8_t *>(counts);
    F.rgba = reinterpret_cast<uint32_t *>(rgba);
    F.hist_bins = reinterpret_cast<uint32_t *>(hist);
    cudaError_t e = launch_coords(nullptr, &F, 1, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "coords kernel launch");
    // The array keeps the previous call's contents: launch_frame clears the
    // work counter and status word (the 16 bytes after the tables) and the
    // histogram with cudaMemsetAsync, and the tables were just rewritten.
    return launch_frame(F, prec, palette, base + coord_pad, st, nullptr);
}
