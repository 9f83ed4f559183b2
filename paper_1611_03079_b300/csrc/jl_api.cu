// C ABI entry points of libjl.so for single frames (include/jl.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>

#include "jl_internal.h"

namespace jl {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(m);
    return e == cudaErrorMemoryAllocation ? JL_ENOMEM : JL_ECUDA;
}

// Built-in palette: a cosine gradient over entries 0..254 and opaque black at
// 255 (points that never escaped).  Channel c of entry k is
// round(255 * (0.5 + 0.5 cos(2 pi (k/254 + phase_c)))), phases 0, 1/3, 2/3.
static void make_default_palette(uint8_t *out)
{
    const double two_pi = 6.283185307179586;
    const double phase[3] = {0.0, 1.0 / 3.0, 2.0 / 3.0};
    for (int k = 0; k < 255; ++k) {
        double t = k / 254.0;
        for (int c = 0; c < 3; ++c) {
            double v = 0.5 + 0.5 * cos(two_pi * (t + phase[c]));
            long q = lround(255.0 * v);
            out[4 * k + c] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
        }
        out[4 * k + 3] = 255;
    }
    out[4 * 255 + 0] = 0;
    out[4 * 255 + 1] = 0;
    out[4 * 255 + 2] = 0;
    out[4 * 255 + 3] = 255;
}

int default_palette_bytes(uint8_t *out)
{
    make_default_palette(out);
    return JL_OK;
}

static bool finite4(const jl_rect &r)
{
    return isfinite(r.xmin) && isfinite(r.xmax) && isfinite(r.ymin) && isfinite(r.ymax);
}

int select_precision(const jl_rect &r, int W, int H)

{
    if (!finite4(r) || !(r.xmin < r.xmax) || !(r.ymin < r.ymax) || W < 1 || H < 1)
        return -1;
    const double dx = (r.xmax - r.xmin) / (double)W;
    const double dy = (r.ymax - r.ymin) / (double)H;
    double m = fabs(r.xmin);
    m = fmax(m, fabs(r.xmax));
    m = fmax(m, fabs(r.ymin));
    m = fmax(m, fabs(r.ymax));
    const float mf = (float)m;
    const float ulp = nextafterf(mf, INFINITY) - mf;
    return (fmin(dx, dy) < 1000.0 * (double)ulp) ? JL_FP64 : JL_FP32;
}

// Validates a frame request and fills the device descriptor (pointers to the
// outputs and coordinate tables are filled by the caller).
int make_frame(double cr, double ci, const jl_rect &rect, int W, int H, int max_iter, int precision, int mode,
               int count_type, bool has_counts, bool has_rgba, bool has_hist, Frame *F, int *prec_out,
               int chunk_len)
{
    if (W < 1 || H < 1 || W > 65536 || H > 65536 || (int64_t)W * (int64_t)H >= (1ll << 31))
        return fail(JL_EINVAL, "width/height out of range (1..65536 each, W*H < 2^31)");
    if (max_iter < 1 || max_iter > 65535)
        return fail(JL_EINVAL, "max_iter out of range (1..65535)");
    if (!finite4(rect) || !(rect.xmin < rect.xmax) || !(rect.ymin < rect.ymax))
        return fail(JL_EINVAL, "rect must be finite with xmin < xmax and ymin < ymax");
    if (mode != JL_JULIA && mode != JL_MANDELBROT)
        return fail(JL_EINVAL, "mode must be JL_JULIA or JL_MANDELBROT");
    if (mode == JL_JULIA && (!isfinite(cr) || !isfinite(ci)))
        return fail(JL_EINVAL, "C must be finite");
    if (precision != JL_FP32 && precision != JL_FP64 && precision != JL_AUTO)
        return fail(JL_EINVAL, "precision must be JL_FP32, JL_FP64 or JL_AUTO");
    if (count_type != JL_COUNT_NONE && count_type != JL_COUNT_U8 && count_type != JL_COUNT_U16)
        return fail(JL_EINVAL, "count_type must be JL_COUNT_NONE, JL_COUNT_U8 or JL_COUNT_U16");
    if (count_type == JL_COUNT_U8 && max_iter > 255)
        return fail(JL_EINVAL, "JL_COUNT_U8 requires max_iter <= 255");
    if ((count_type == JL_COUNT_NONE) == has_counts)
        return fail(JL_EINVAL, "counts must be NULL exactly when count_type is JL_COUNT_NONE");
    if (!has_counts && !has_rgba && !has_hist)
        return fail(JL_EINVAL, "no output requested");
    int prec = precision == JL_AUTO ? select_precision(rect, W, H) : precision;
    if (prec < 0)
        return fail(JL_EINVAL, "invalid rect for precision selection");

    memset(F, 0, sizeof(*F));
    F->cr = mode == JL_JULIA ? cr : 0.0;
    F->ci = mode == JL_JULIA ? ci : 0.0;
    F->cr32 = (float)F->cr;  // round to nearest even, as the binary32 path requires
    F->ci32 = (float)F->ci;
    F->xmin = rect.xmin;
    F->ymin = rect.ymin;
    F->dx = (rect.xmax - rect.xmin) / (double)W;
    F->dy = (rect.ymax - rect.ymin) / (double)H;
    F->W = W;
    F->H = H;
    F->max_iter = max_iter;
    F->mode = mode;
    F->count_type = count_type;
    if (chunk_len < 16 || chunk_len > 1024)
        return fail(JL_EINVAL, "chunk_len must be 16..1024");
    // Work chunks: row segments of chunk_len pixels, or whole rows grouped
    // k = chunk_len / W at a time for narrow frames.  For the grouped form the
    // row of pixel o < k*W <= 1024 is (o * ceil(2^20 / W)) >> 20, exact because
    // the excess o * (ceil(2^20/W) - 2^20/W) / 2^20 < 2^-10 <= 1/W.
    F->chunk_len = chunk_len;
    if (W < chunk_len && chunk_len / W > 1) {
        F->rows_per_chunk = chunk_len / W;
        F->span_magic = (uint32_t)(((1u << 20) + (uint32_t)W - 1u) / (uint32_t)W);
        F->chunks_per_row = 1;
        F->chunk_count = (H + F->rows_per_chunk - 1) / F->rows_per_chunk;
    } else {
        F->rows_per_chunk = 1;
        F->span_magic = 0;
        F->chunks_per_row = (W + chunk_len - 1) / chunk_len;
        F->chunk_count = H * F->chunks_per_row;
    }
    F->tiles_x = (W + 31) / 32;
    F->tile_count = F->tiles_x * ((H + 31) / 32);
    // t / tiles_x = (t * m) >> 40 with m = floor(2^40 / tiles_x) + 1 is exact for
    // t < 2^40 / tiles_x; here t < tile_count <= 2^22 and tiles_x <= 2^11.
    F->tiles_x_magic = (1ull << 40) / (uint64_t)F->tiles_x + 1ull;
    F->tile_begin = 0;
    F->precision = prec;
    F->colour_magic = (1ull << 40) / (uint64_t)max_iter + 1ull;
    if (prec == JL_FP64 && mode == JL_JULIA) {
        F->cert_ec = cert_error_constant(F->cr, F->ci, F->cr32, F->ci32);
        cert2_frame_constants(F->cr, F->ci, F->cr32, F->ci32, &F->cr_lo32, &F->ci_lo32, &F->cert2_kc);
    }
    // Monotone escape is proven for |C| <= 2 - 2^-12 (Julia); Mandelbrot pixels
    // are classified one by one in the kernel.  |C|^2 < 3.99 is inside that.
    if (mode == JL_JULIA) {
        double c2;
        if (prec == JL_FP32) {
            double fr = (double)(float)cr, fi = (double)(float)ci;
            c2 = fr * fr + fi * fi;
        } else {
            c2 = cr * cr + ci * ci;
        }
        F->safe = c2 < 3.99 ? 1 : 0;
    } else {
        F->safe = 1;
    }
    *prec_out = prec;
    return JL_OK;
}

// Launches the escape kernel of one frame whose coordinate tables (F.xs,
// F.ys) are already filled: clears the 48-byte control block `ctl` (work
// counter, status, the certified passes' list counts and list counters) and
// the histogram, runs the kernel and finalises the histogram.  A binary64
// frame with binary32 tables and a list of cert_cap >= W * H entries takes the
// certified binary32 pass (and the double-float pass with a second list).
// All pointers are device pointers.
int launch_frame(Frame &F, int prec, const uint8_t *palette, void *ctl, cudaStream_t st, const Variant *vopt,
                 uint64_t *cert_list, int64_t cert_cap, uint64_t *cert_list2)
{
    unsigned long long *counter = static_cast<unsigned long long *>(ctl);
    int32_t *status = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ctl) + 8);
    cudaError_t e = cudaMemsetAsync(ctl, 0, 48, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(counter)");
    if (F.hist_bins) {
        e = cudaMemsetAsync(F.hist_bins, 0, ((size_t)F.max_iter + 1) * 4, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync(hist)");
    }
    EscapeArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = nullptr;
    a.n_frames = 1;
    a.hist_smem = (F.hist_bins && F.max_iter + 1 <= 4096) ? 1 : 0;
    a.total_chunks = F.chunk_count;
    a.total_tiles = F.tile_count;
    a.chunk_counter = counter;
    a.status = status;
    a.cycle_budget = 0;
    if (prec == JL_FP64 && cert_list && cert_cap >= (int64_t)F.W * F.H && F.xs32 && F.ys32 && F.xs32lo &&
        F.ys32lo) {
        a.cert_list = cert_list;
        a.cert_cap = cert_cap;
        a.cert_count = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(ctl) + 16);
        a.list_counter = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(ctl) + 24);
        if (cert_list2) {
            a.cert_list2 = cert_list2;
            a.cert_count2 = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(ctl) + 32);
            a.list2_counter = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(ctl) + 40);
        }
    } else {
        F.xs32 = nullptr;
        F.ys32 = nullptr;
        F.xs32lo = nullptr;
        F.ys32lo = nullptr;
    }
    uint8_t pal[1024];
    if (palette)
        memcpy(pal, palette, 1024);
    else
        make_default_palette(pal);
    memcpy(a.palette, pal, 1024);
    a.single = F;
    const int sms = device_sm_count();
    if (sms <= 0)
        return fail(JL_EUNSUPPORTED, "no CUDA device");
    Variant v = vopt ? *vopt : tuned_variant(prec, F.max_iter);
    e = launch_escape(a, prec, v, sms, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "escape kernel launch");
    if (F.hist_bins) {
        e = launch_hist_finalize(nullptr, &F, 1, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "histogram finalize launch");
    }
    return JL_OK;
}

// Renders one frame whose descriptor is complete except for scratch-backed
// fields; all pointers in F are device pointers.
int render_frame(Frame &F, int prec, const uint8_t *palette, cudaStream_t st, const Variant *vopt)
{
    const size_t esz = prec == JL_FP64 ? 8 : 4;
    const size_t coord_bytes = ((size_t)F.W + (size_t)F.H) * esz;
    const size_t coord_pad = (coord_bytes + 255) & ~(size_t)255;
    // binary64: binary32 tables and the two lists of the certified passes (8 B per pixel each)
    const size_t c32_pad = prec == JL_FP64 ? ((((size_t)F.W + (size_t)F.H) * 8 + 255) & ~(size_t)255) : 0;
    const size_t list_bytes = prec == JL_FP64 ? (size_t)F.W * (size_t)F.H * 16 : 0;
    const size_t scratch_bytes = coord_pad + 256 + c32_pad + list_bytes;
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, scratch_bytes, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(scratch)");
    uint8_t *base = static_cast<uint8_t *>(scratch);
    F.xs = base;
    F.ys = base + (size_t)F.W * esz;
    uint64_t *list = nullptr;
    if (prec == JL_FP64) {
        F.xs32 = reinterpret_cast<float *>(base + coord_pad + 256);
        F.ys32 = F.xs32 + F.W;
        F.xs32lo = F.ys32 + F.H;
        F.ys32lo = F.xs32lo + F.W;
        list = reinterpret_cast<uint64_t *>(base + coord_pad + 256 + c32_pad);
    }
    int rc = JL_OK;
    e = launch_coords(nullptr, &F, 1, st);
    if (e != cudaSuccess)
        rc = cuda_fail(e, "coords kernel launch");
    if (rc == JL_OK)
        rc = launch_frame(F, prec, palette, base + coord_pad, st, vopt, list, (int64_t)F.W * F.H,
                          list ? list + (size_t)F.W * F.H : nullptr);
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (rc == JL_OK && e2 != cudaSuccess)
        rc = cuda_fail(e2, "cudaFreeAsync(scratch)");
    return rc;
}

}  // namespace jl

using namespace jl;

extern "C" {

const char *jl_last_error(void) { return g_last_error.c_str(); }

const char *jl_version(void) { return "jl 0.1 (sm_103a)"; }

int jl_select_precision(jl_rect rect, int32_t width, int32_t height)
{
    return select_precision(rect, width, height);
}

int jl_variant_list(int32_t precision, int32_t *pairs, int32_t cap)
{
    if (precision != JL_FP32 && precision != JL_FP64)
        return fail(-1, "precision must be JL_FP32 or JL_FP64");
    return variant_list(precision, pairs, cap < 0 ? 0 : cap);
}

int jl_selftest_double(const double *in, double *out, int32_t n, void *stream)
{
    if (!in || !out || n < 1)
        return fail(JL_EINVAL, "invalid arguments");
    cudaError_t e = launch_dbl2(in, out, n, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "jl_selftest_double");
}

int jl_default_palette(uint8_t *out)
{
    if (!out)
        return fail(JL_EINVAL, "out must not be NULL");
    make_default_palette(out);
    return JL_OK;
}

int jl_render(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
              int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
              const uint8_t *palette, float *hist, void *stream)
{
    Frame F;
    int prec = 0;
    int rc = make_frame(cr, ci, rect, width, height, max_iter, precision, mode, count_type, counts != nullptr,
                        rgba != nullptr, hist != nullptr, &F, &prec);
    if (rc != JL_OK)
        return rc;
    F.counts = static_cast<uint8_t *>(counts);
    F.rgba = reinterpret_cast<uint32_t *>(rgba);
    F.hist_bins = reinterpret_cast<uint32_t *>(hist);
    return render_frame(F, prec, palette, static_cast<cudaStream_t>(stream), nullptr);
}

// Same as jl_render with an explicit kernel variant (autotuner and tests).
int jl_render_variant(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
                      int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
                      const uint8_t *palette, float *hist, int32_t ppt, int32_t unroll, int32_t threads,
                      int32_t ctas_per_sm, void *stream)
{
    Frame F;
    int prec = 0;
    int rc = make_frame(cr, ci, rect, width, height, max_iter, precision, mode, count_type, counts != nullptr,
                        rgba != nullptr, hist != nullptr, &F, &prec);
    if (rc != JL_OK)
        return rc;
    if (!variant_supported(prec, ppt, unroll))
        return fail(JL_EINVAL, "unsupported (ppt, unroll) for this precision");
    if (ppt == 0)
        threads = 256;  // the static kernel has a fixed CTA shape
    if (threads < 32 || threads > 256 || (threads & 31))
        return fail(JL_EINVAL, "threads must be a multiple of 32 in 32..256");
    if (ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(JL_EINVAL, "ctas_per_sm must be 0 (occupancy maximum) .. 32");
    F.counts = static_cast<uint8_t *>(counts);
    F.rgba = reinterpret_cast<uint32_t *>(rgba);
    F.hist_bins = reinterpret_cast<uint32_t *>(hist);
    Variant v{ppt, unroll, threads, ctas_per_sm};
    return render_frame(F, prec, palette, static_cast<cudaStream_t>(stream), &v);
}

int jl_render_to_host(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
                      int32_t precision, int32_t mode, int32_t count_type, void *counts_host,
                      uint8_t *rgba_host, const uint8_t *palette, float *hist_host, void *stream)
{
    Frame F;
    int prec = 0;
    int rc = make_frame(cr, ci, rect, width, height, max_iter, precision, mode, count_type,
                        counts_host != nullptr, rgba_host != nullptr, hist_host != nullptr, &F, &prec);
    if (rc != JL_OK)
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t npix = (size_t)width * (size_t)height;
    const size_t cbytes = counts_host ? npix * (count_type == JL_COUNT_U8 ? 1 : 2) : 0;
    const size_t rbytes = rgba_host ? npix * 4 : 0;
    const size_t hbytes = hist_host ? ((size_t)max_iter + 1) * 4 : 0;
    auto pad = [](size_t b) { return (b + 255) & ~(size_t)255; };
    void *dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, pad(cbytes) + pad(rbytes) + pad(hbytes) + 256, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(outputs)");
    uint8_t *b = static_cast<uint8_t *>(dev);
    F.counts = counts_host ? b : nullptr;
    F.rgba = rgba_host ? reinterpret_cast<uint32_t *>(b + pad(cbytes)) : nullptr;
    F.hist_bins = hist_host ? reinterpret_cast<uint32_t *>(b + pad(cbytes) + pad(rbytes)) : nullptr;
    rc = render_frame(F, prec, palette, st, nullptr);
    if (rc == JL_OK && counts_host) {
        e = cudaMemcpyAsync(counts_host, F.counts, cbytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(counts)");
    }
    if (rc == JL_OK && rgba_host) {
        e = cudaMemcpyAsync(rgba_host, F.rgba, rbytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(rgba)");
    }
    if (rc == JL_OK && hist_host) {
        e = cudaMemcpyAsync(hist_host, F.hist_bins, hbytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(hist)");
    }
    e = cudaFreeAsync(dev, st);
    if (rc == JL_OK && e != cudaSuccess)
        rc = cuda_fail(e, "cudaFreeAsync(outputs)");
    e = cudaStreamSynchronize(st);
    if (rc == JL_OK && e != cudaSuccess)
        rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // extern "C"
