// Autotuner for the escape kernel's launch shape: pixels per thread (ILP
// slots), steps per block, threads per CTA.  Every supported candidate is
// timed with CUDA events on a calibration set of frames; the fastest is kept
// in a per-process table keyed by (device, precision, iteration-limit
// bucket) that jl_render and batch plans consult.  The table can be saved to
// and loaded from a small text file.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "jl_internal.h"

namespace jl {

static constexpr int kTuneDevices = 64;
static constexpr int kBuckets = 4;  // limit <= 128, <= 1024, <= 8192, larger

struct TuneEntry {
    bool valid = false;
    Variant v{};
    double ms = 0.0;
};

static std::mutex g_tune_mu;
static TuneEntry g_tune[kTuneDevices][2][kBuckets];

static int bucket_of(int max_iter)
{
    if (max_iter <= 128)
        return 0;
    if (max_iter <= 1024)
        return 1;
    if (max_iter <= 8192)
        return 2;
    return 3;
}

Variant tuned_variant(int precision, int max_iter)
{
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kTuneDevices) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        const TuneEntry &t = g_tune[dev][precision ? 1 : 0][bucket_of(max_iter)];
        if (t.valid)
            return t.v;
    }
    return default_variant(precision, max_iter);
}

}  // namespace jl

using namespace jl;

extern "C" int jl_render_variant(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
                                 int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
                                 const uint8_t *palette, float *hist, int32_t ppt, int32_t unroll, int32_t threads,
                                 int32_t ctas_per_sm, void *stream);

extern "C" {

int jl_autotune(int32_t precision, int32_t max_iter, const jl_frame *calib, int32_t n_calib, int32_t reps,
                jl_tune_result *out)
{
    if (precision != JL_FP32 && precision != JL_FP64)
        return fail(JL_EINVAL, "precision must be JL_FP32 or JL_FP64");
    if (max_iter < 1 || max_iter > 65535)
        return fail(JL_EINVAL, "max_iter out of range");
    if (reps < 1)
        reps = 3;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kTuneDevices)
        return fail(JL_EUNSUPPORTED, "device index beyond the tuning table");

    // Calibration set: the caller's frames, else a built-in pair (a connected
    // Julia set and the Mandelbrot plane) at 1024 x 1024.
    std::vector<jl_frame> set;
    if (calib && n_calib > 0) {
        set.assign(calib, calib + n_calib);
    } else {
        jl_frame a;
        memset(&a, 0, sizeof(a));
        a.cr = -0.7269;
        a.ci = 0.1889;
        a.rect = jl_rect{-1.6, 1.6, -1.6, 1.6};
        a.width = a.height = 1024;
        a.mode = JL_JULIA;
        set.push_back(a);
        jl_frame m = a;
        m.rect = jl_rect{-2.5, 1.0, -1.75, 1.75};
        m.mode = JL_MANDELBROT;
        set.push_back(m);
    }
    size_t max_pix = 0;
    for (const jl_frame &f : set) {
        if (f.width < 1 || f.height < 1 || f.width > 65536 || f.height > 65536)
            return fail(JL_EINVAL, "calibration frame size out of range");
        max_pix = std::max(max_pix, (size_t)f.width * (size_t)f.height);
    }
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    void *buf = nullptr;
    e = cudaMalloc(&buf, max_pix * 4);
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        return cuda_fail(e, "cudaMalloc(tuning output)");
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);

    int32_t pairs[64];
    const int np = variant_list(precision, pairs, 32);
    const int thread_opts[2] = {128, 256};
    TuneEntry best;
    int rc = JL_OK;
    int tried = 0;
    std::vector<Variant> cands;
    for (int pi = 0; pi < np; ++pi) {
        for (int ti = 0; ti < 2; ++ti) {
            Variant v{pairs[2 * pi], pairs[2 * pi + 1], thread_opts[ti], 0};
            if (v.ppt == 0 && ti == 1)
                continue;  // the static kernel has one CTA shape
            cands.push_back(v);
        }
    }
    for (size_t ci = 0; ci < cands.size() && rc == JL_OK; ++ci) {
        {
            const Variant v = cands[ci];
            float total = 0.f;
            for (int r = 0; r <= reps && rc == JL_OK; ++r) {  // r == 0 warms up
                cudaEventRecord(t0, st);
                for (const jl_frame &f : set) {
                    rc = jl_render_variant(f.cr, f.ci, f.rect, f.width, f.height, max_iter, precision, f.mode,
                                           JL_COUNT_NONE, nullptr, static_cast<uint8_t *>(buf), nullptr, nullptr,
                                           v.ppt, v.unroll, v.threads, v.ctas_per_sm, st);
                    if (rc != JL_OK)
                        break;
                }
                cudaEventRecord(t1, st);
                e = cudaEventSynchronize(t1);
                if (rc == JL_OK && e != cudaSuccess)
                    rc = cuda_fail(e, "tuning run");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (r > 0)
                    total += ms;
            }
            if (rc != JL_OK)
                break;
            const double mean = total / reps;
            ++tried;
            // candidates are listed simplest first (the static tile kernel); a
            // later one must win by more than 1 % (run-to-run noise) to replace it
            if (!best.valid || mean < best.ms * 0.99) {
                best.valid = true;
                best.v = v;
                best.ms = mean;
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(buf);
    cudaStreamDestroy(st);
    if (rc != JL_OK)
        return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[dev][precision][bucket_of(max_iter)] = best;
    }
    if (out) {
        out->ppt = best.v.ppt;
        out->unroll = best.v.unroll;
        out->threads = best.v.threads;
        out->ctas_per_sm = best.v.ctas_per_sm;
        out->ms = best.ms;
        out->candidates = tried;
    }
    return JL_OK;
}

int jl_tune_get(int32_t precision, int32_t max_iter, jl_tune_result *out)
{
    if (!out || (precision != JL_FP32 && precision != JL_FP64) || max_iter < 1)
        return fail(JL_EINVAL, "invalid arguments");
    Variant v = tuned_variant(precision, max_iter);
    int dev = 0;
    cudaGetDevice(&dev);
    bool tuned = false;
    double ms = 0.0;
    if (dev >= 0 && dev < kTuneDevices) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tuned = g_tune[dev][precision][bucket_of(max_iter)].valid;
        ms = g_tune[dev][precision][bucket_of(max_iter)].ms;
    }
    out->ppt = v.ppt;
    out->unroll = v.unroll;
    out->threads = v.threads;
    out->ctas_per_sm = v.ctas_per_sm;
    out->ms = ms;
    out->candidates = tuned ? 1 : 0;
    return JL_OK;
}

int jl_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &d : g_tune)
        for (auto &p : d)
            for (auto &b : p)
                b = TuneEntry{};
    return JL_OK;
}

// Text format, one line per entry:  device precision bucket ppt unroll threads ctas_per_sm ms
int jl_tune_save(const char *path)
{
    if (!path)
        return fail(JL_EINVAL, "path must not be NULL");
    FILE *fp = fopen(path, "w");
    if (!fp)
        return fail(JL_EINVAL, std::string("cannot open ") + path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    fprintf(fp, "# jl tuning table v3: device precision bucket ppt unroll threads ctas_per_sm ms\n");
    for (int d = 0; d < kTuneDevices; ++d)
        for (int p = 0; p < 2; ++p)
            for (int b = 0; b < kBuckets; ++b) {
                const TuneEntry &t = g_tune[d][p][b];
                if (t.valid)
                    fprintf(fp, "%d %d %d %d %d %d %d %.6f\n", d, p, b, t.v.ppt, t.v.unroll, t.v.threads,
                            t.v.ctas_per_sm, t.ms);
            }
    fclose(fp);
    return JL_OK;
}

int jl_tune_load(const char *path)
{
    if (!path)
        return fail(JL_EINVAL, "path must not be NULL");
    FILE *fp = fopen(path, "r");
    if (!fp)
        return fail(JL_EINVAL, std::string("cannot open ") + path);
    char line[256];
    int loaded = 0;
    int rc = JL_OK;
    std::vector<std::pair<int, TuneEntry>> entries;
    while (fgets(line, sizeof(line), fp)) {
        if (line[0] == '#' || line[0] == '\n')
            continue;
        int d, p, b, ppt, un, th, cps;
        double ms;
        if (sscanf(line, "%d %d %d %d %d %d %d %lf", &d, &p, &b, &ppt, &un, &th, &cps, &ms) != 8 || d < 0 ||
            d >= kTuneDevices || p < 0 || p > 1 || b < 0 || b >= kBuckets || !variant_supported(p, ppt, un) ||
            th < 32 || th > 256 || (th & 31) || cps < 0 || cps > 32) {
            rc = fail(JL_EINVAL, std::string("malformed tuning line: ") + line);
            break;
        }
        TuneEntry t;
        t.valid = true;
        t.v = Variant{ppt, un, th, cps};
        t.ms = ms;
        entries.push_back({(d * 2 + p) * kBuckets + b, t});
    }
    fclose(fp);
    if (rc != JL_OK)
        return rc;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &kv : entries) {
        const int idx = kv.first;
        g_tune[idx / (2 * kBuckets)][(idx / kBuckets) % 2][idx % kBuckets] = kv.second;
        ++loaded;
    }
    return loaded >= 0 ? JL_OK : JL_EINVAL;
}

}  // extern "C"
