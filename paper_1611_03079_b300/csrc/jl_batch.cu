// Batched rendering: many frames (different C, view, size, limit, mode and
// precision) in one CUDA-graph launch of persistent escape kernels
// (paper Sec. 3: parameter paths animated in real time; Sec. 2: the
// escape-time kernel itself lives in jl_escape.cu).
//
// A plan resolves every frame's precision, builds the device frame tables and
// the work-unit -> frame table, and captures one graph: reset of the work
// counters and status word, the coordinate tables of every frame, zeroing of
// the histogram bins, the binary32 and binary64 persistent escape kernels on
// two forked branches (they run concurrently, so binary32 work fills the issue
// slots the narrow binary64 pipe leaves idle), and the histogram finalisation.
// Launching the plan replays the graph; nothing is allocated per launch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <algorithm>
#include <vector>

#include "jl_internal.h"

struct jl_batch {
    int device = -1;
    int n = 0;
    std::vector<int32_t> prec;             // resolved precision of every frame (input order)
    std::vector<int64_t> pixels;           // per group
    jl::Frame *frames_dev[2] = {nullptr, nullptr};
    int32_t *chunk_frame_dev[2] = {nullptr, nullptr};  // chunk -> frame (lane-refill kernel)
    int32_t *tile_dev[2] = {nullptr, nullptr};         // tile kernels: tile -> frame, then tile -> index in frame
    bool tuned[2] = {false, false};                    // variant chosen by timing the plan's own frames
    int64_t tiles[2] = {0, 0};
    int n_group[2] = {0, 0};
    int64_t chunks[2] = {0, 0};
    void *coords_dev = nullptr;
    uint64_t *list_dev = nullptr;          // binary64 group: the certified passes' two lists (8 B per pixel each)
    // control words, zeroed per launch: work counters of the two groups (0, 8),
    // status (16), the binary32 pass's list count (32), the binary64 kernel's
    // list counter (40), the binary64 kernel's iterations (48), the
    // double-float pass's list count (56), its counter on the first list (64),
    // the iterations of the pixels it settles (72), and the tests decided by the
    // binary32 pass (80) and the double-float pass (88)
    uint8_t *ctl_dev = nullptr;
    // opts.variant_flags bit 3: timing events recorded inside the graph around
    // the binary32 kernel (0, 1) and the binary64 kernels (2, 3 after the
    // binary32 pass, 5 after the double-float pass, 4)
    bool phases = false, cert_used = false, cert2_used = false;
    cudaEvent_t ph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t s0 = nullptr, s1 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t certs_done = nullptr;      // the binary64 group's certified passes are done
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    jl::Variant variant[2];
    bool any_hist = false;
};

namespace jl {

static void destroy_plan(jl_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    for (int g = 0; g < 2; ++g) {
        if (b->frames_dev[g])
            cudaFree(b->frames_dev[g]);
        if (b->chunk_frame_dev[g])
            cudaFree(b->chunk_frame_dev[g]);
        if (b->tile_dev[g])
            cudaFree(b->tile_dev[g]);
    }
    if (b->coords_dev)
        cudaFree(b->coords_dev);
    if (b->list_dev)
        cudaFree(b->list_dev);
    if (b->ctl_dev)
        cudaFree(b->ctl_dev);
    for (cudaEvent_t &ev : b->ph)
        if (ev)
            cudaEventDestroy(ev);
    if (b->fork)
        cudaEventDestroy(b->fork);
    if (b->join)
        cudaEventDestroy(b->join);
    if (b->certs_done)
        cudaEventDestroy(b->certs_done);
    if (b->s0)
        cudaStreamDestroy(b->s0);
    if (b->s1)
        cudaStreamDestroy(b->s1);
    delete b;
}



}  // namespace jl

using namespace jl;

extern "C" {

int jl_batch_create(const jl_frame *frames, int32_t n, void *counts_base, uint8_t *rgba_base, float *hist_base,
                    const uint8_t *palette, const jl_batch_opts *opts, jl_batch **out)
{
    if (!out)
        return fail(JL_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (!frames || n < 1)
        return fail(JL_EINVAL, "need at least one frame");
    jl_batch_opts o;
    memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    const int chunk_len = o.chunk_len ? o.chunk_len : 512;
    if (o.cycle_budget < 0)
        return fail(JL_EINVAL, "cycle_budget must be >= 0");

    // ---- validate and describe every frame ----
    std::vector<Frame> host[2];
    std::vector<int32_t> prec(n);
    std::vector<int> max_iter_max(2, 1);
    bool any_hist = false;
    for (int f = 0; f < n; ++f) {
        const jl_frame &q = frames[f];
        const bool hc = q.counts_offset >= 0, hr = q.rgba_offset >= 0, hh = q.hist_offset >= 0;
        if ((hc && !counts_base) || (hr && !rgba_base) || (hh && !hist_base))
            return fail(JL_EINVAL, "frame " + std::to_string(f) + ": output offset given but base pointer is NULL");
        if (hh && (q.hist_offset & 3))
            return fail(JL_EINVAL, "frame " + std::to_string(f) + ": hist_offset must be a multiple of 4");
        if (hr && (q.rgba_offset & 3))
            return fail(JL_EINVAL, "frame " + std::to_string(f) + ": rgba_offset must be a multiple of 4");
        if (hc && q.count_type == JL_COUNT_U16 && (q.counts_offset & 1))
            return fail(JL_EINVAL, "frame " + std::to_string(f) + ": uint16 counts_offset must be even");
        Frame F;
        int p = 0;
        int rc = make_frame(q.cr, q.ci, q.rect, q.width, q.height, q.max_iter, q.precision, q.mode, q.count_type,
                            hc, hr, hh, &F, &p, chunk_len);
        if (rc != JL_OK)
            return fail(rc, "frame " + std::to_string(f) + ": " + jl_last_error());
        F.counts = hc ? static_cast<uint8_t *>(counts_base) + q.counts_offset : nullptr;
        F.rgba = hr ? reinterpret_cast<uint32_t *>(rgba_base + q.rgba_offset) : nullptr;
        F.hist_bins = hh ? reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(hist_base) + q.hist_offset)
                         : nullptr;
        any_hist |= hh;
        prec[f] = p;
        if (q.max_iter > max_iter_max[p])
            max_iter_max[p] = q.max_iter;
        host[p].push_back(F);
    }

    jl_batch *b = new jl_batch();
    b->n = n;
    b->prec = prec;
    b->any_hist = any_hist;
    b->pixels.assign(2, 0);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        destroy_plan(b);
        return cuda_fail(e, "cudaGetDevice");
    }
    int rc = JL_OK;
    do {
        // ---- coordinate tables (one allocation, 256-byte aligned pieces) ----
        // (binary64 frames: also their binary32 roundings for the certified pass)
        size_t coord_bytes = 0;
        for (int g = 0; g < 2; ++g)
            for (const Frame &F : host[g])
                coord_bytes += (((size_t)F.W * (g ? 8 : 4) + 255) & ~(size_t)255) +
                               (((size_t)F.H * (g ? 8 : 4) + 255) & ~(size_t)255) +
                               (g ? 2 * ((((size_t)F.W * 4 + 255) & ~(size_t)255) +
                                         (((size_t)F.H * 4 + 255) & ~(size_t)255))
                                  : 0);
        e = cudaMalloc(&b->coords_dev, coord_bytes ? coord_bytes : 256);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(coordinate tables)"); break; }
        size_t off = 0;
        for (int g = 0; g < 2; ++g) {
            int64_t chunk = 0, tile = 0;
            for (Frame &F : host[g]) {
                F.tile_begin = tile;
                tile += F.tile_count;
                const size_t es = g ? 8 : 4;
                F.xs = static_cast<uint8_t *>(b->coords_dev) + off;
                off += ((size_t)F.W * es + 255) & ~(size_t)255;
                F.ys = static_cast<uint8_t *>(b->coords_dev) + off;
                off += ((size_t)F.H * es + 255) & ~(size_t)255;
                if (g) {
                    F.xs32 = reinterpret_cast<const float *>(static_cast<uint8_t *>(b->coords_dev) + off);
                    off += ((size_t)F.W * 4 + 255) & ~(size_t)255;
                    F.ys32 = reinterpret_cast<const float *>(static_cast<uint8_t *>(b->coords_dev) + off);
                    off += ((size_t)F.H * 4 + 255) & ~(size_t)255;
                    F.xs32lo = reinterpret_cast<const float *>(static_cast<uint8_t *>(b->coords_dev) + off);
                    off += ((size_t)F.W * 4 + 255) & ~(size_t)255;
                    F.ys32lo = reinterpret_cast<const float *>(static_cast<uint8_t *>(b->coords_dev) + off);
                    off += ((size_t)F.H * 4 + 255) & ~(size_t)255;
                }
                F.chunk_begin = chunk;
                chunk += F.chunk_count;
                b->pixels[g] += (int64_t)F.W * F.H;
            }
            b->chunks[g] = chunk;
            b->tiles[g] = tile;
            b->n_group[g] = (int)host[g].size();
        }
        e = cudaMalloc(&b->ctl_dev, 256);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(control words)"); break; }
        if (b->pixels[1] > 0) {
            e = cudaMalloc(&b->list_dev, (size_t)b->pixels[1] * sizeof(uint64_t) * 2);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(certified pass list)"); break; }
        }
        e = cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&b->s1, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->certs_done, cudaEventDisableTiming);
        b->phases = (o.variant_flags & 8) != 0;
        for (int k = 0; k < 6 && e == cudaSuccess && b->phases; ++k)
            e = cudaEventCreate(&b->ph[k]);
        if (e != cudaSuccess) { rc = cuda_fail(e, "stream/event creation"); break; }

        for (int g = 0; g < 2 && rc == JL_OK; ++g) {
            if (host[g].empty())
                continue;
            // kernel variant: explicit option, else the tuned/default one
            const int pp = g ? o.fp64_ppt : o.fp32_ppt;
            const int uu = g ? o.fp64_unroll : o.fp32_unroll;
            const int tt = g ? o.fp64_threads : o.fp32_threads;
            const bool explicit_variant = pp || uu || ((o.variant_flags >> g) & 1);
            Variant v = tuned_variant(g, max_iter_max[g]);
            if (explicit_variant) {
                if (!variant_supported(g, pp, uu)) { rc = fail(JL_EINVAL, "unsupported (ppt, unroll) option"); break; }
                v.ppt = pp;
                v.unroll = uu;
            }
            if (tt) {
                if (tt < 32 || tt > 256 || (tt & 31)) { rc = fail(JL_EINVAL, "threads option must be 32..256, multiple of 32"); break; }
                v.threads = tt;
            }
            b->variant[g] = v;
            if (v.ppt == 0 && b->tiles[g] > 0x7fffffffll) { rc = fail(JL_EINVAL, "too many tiles for the static kernel"); break; }
            const size_t nb = host[g].size() * sizeof(Frame);
            e = cudaMalloc(&b->frames_dev[g], nb);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(frame table)"); break; }
            e = cudaMemcpy(b->frames_dev[g], host[g].data(), nb, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpy(frame table)"); break; }
            // Work tables, both kinds (a tuned plan may try either).  Lane-refill
            // kernel: chunk -> frame, in frame order.  Tile kernels: 32x32 tiles
            // of the frames with the highest limit first, each limit's frames
            // interleaved (round-robin over the frames that still have tiles),
            // then each tile's index within its frame.  Warps claiming work
            // meet the far field and the costly regions of several frames alike
            // rather than one frame's far field at a time (cheap tiles claimed in
            // a burst make the launch counter the bottleneck), and the launch
            // ends on cheap tiles rather than on a few long ones; the certified
            // pass's list, appended in this order, then starts with the
            // long-lived pixels, so the double-float pass ends on short ones
            // (sweep step 9.51 -> 9.35 ms against one round-robin over all
            // frames; the double-float pass 2.32 -> 2.23 ms).
            {
                std::vector<int32_t> cf((size_t)b->chunks[g]);
                for (size_t f = 0; f < host[g].size(); ++f) {
                    const int64_t begin = host[g][f].chunk_begin;
                    for (int32_t c = 0; c < host[g][f].chunk_count; ++c)
                        cf[(size_t)begin + c] = (int32_t)f;
                }
                e = cudaMalloc(&b->chunk_frame_dev[g], std::max<size_t>(cf.size(), 1) * sizeof(int32_t));
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(chunk table)"); break; }
                e = cudaMemcpy(b->chunk_frame_dev[g], cf.data(), cf.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpy(chunk table)"); break; }
            }
            if (b->tiles[g] <= 0x7fffffffll) {
                const size_t T = (size_t)b->tiles[g];
                std::vector<int32_t> tf(2 * T);
                // frame indices by limit, highest first (stable: input order within a limit)
                std::vector<int32_t> by_lim(host[g].size());
                for (size_t f = 0; f < by_lim.size(); ++f)
                    by_lim[f] = (int32_t)f;
                std::stable_sort(by_lim.begin(), by_lim.end(), [&](int32_t u, int32_t v) {
                    return host[g][u].max_iter > host[g][v].max_iter;
                });
                size_t pos = 0;
                for (size_t g0 = 0; g0 < by_lim.size();) {
                    size_t g1 = g0;
                    int32_t most = 0;
                    while (g1 < by_lim.size() && host[g][by_lim[g1]].max_iter == host[g][by_lim[g0]].max_iter) {
                        most = std::max(most, host[g][by_lim[g1]].tile_count);
                        ++g1;
                    }
                    // round-robin over this limit's frames; frames that run out of
                    // tiles drop out of the rotation
                    std::vector<int32_t> act(by_lim.begin() + (long)g0, by_lim.begin() + (long)g1);
                    for (int32_t k = 0; k < most && !act.empty(); ++k) {
                        size_t keep = 0;
                        for (size_t q = 0; q < act.size(); ++q) {
                            const int32_t f = act[q];
                            tf[pos] = f;
                            tf[T + pos] = k;
                            ++pos;
                            if (k + 1 < host[g][f].tile_count)
                                act[keep++] = f;
                        }
                        act.resize(keep);
                    }
                    g0 = g1;
                }
                e = cudaMalloc(&b->tile_dev[g], std::max<size_t>(tf.size(), 1) * sizeof(int32_t));
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(tile table)"); break; }
                e = cudaMemcpy(b->tile_dev[g], tf.data(), tf.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpy(tile table)"); break; }
            }
            b->tuned[g] = o.tune != 0 && !explicit_variant;
        }
        if (rc != JL_OK)
            break;

        // ---- capture the launch graph ----
        EscapeArgs args[2];
        uint8_t pal[1024];
        if (palette)
            memcpy(pal, palette, 1024);
        else
            default_palette_bytes(pal);
        auto make_args = [&](int g, const Variant &v) {
            EscapeArgs x;
            memset(&x, 0, sizeof(EscapeArgs));
            x.frames = b->frames_dev[g];
            x.chunk_frame = b->chunk_frame_dev[g];
            x.tile_frame = b->tile_dev[g];
            x.tile_local = b->tile_dev[g] ? b->tile_dev[g] + b->tiles[g] : nullptr;
            x.total_tiles = b->tiles[g];
            x.n_frames = b->n_group[g];
            x.hist_smem = 0;
            x.total_chunks = b->chunks[g];
            x.chunk_counter = reinterpret_cast<unsigned long long *>(b->ctl_dev + 8 * g);
            x.status = reinterpret_cast<int32_t *>(b->ctl_dev + 16);
            x.cycle_budget = o.cycle_budget;
            if (g == 1 && b->list_dev && !(o.variant_flags & 4)) {
                x.cert_list = b->list_dev;
                x.cert_cap = b->pixels[1];
                x.cert_count = reinterpret_cast<unsigned long long *>(b->ctl_dev + 32);
                x.list_counter = reinterpret_cast<unsigned long long *>(b->ctl_dev + 40);
                x.list_iters = reinterpret_cast<unsigned long long *>(b->ctl_dev + 48);
                x.cert_steps = reinterpret_cast<unsigned long long *>(b->ctl_dev + 80);
                if (!(o.variant_flags & 16)) {
                    x.cert_list2 = b->list_dev + b->pixels[1];
                    x.cert_count2 = reinterpret_cast<unsigned long long *>(b->ctl_dev + 56);
                    x.list2_counter = reinterpret_cast<unsigned long long *>(b->ctl_dev + 64);
                    x.cert2_iters = reinterpret_cast<unsigned long long *>(b->ctl_dev + 72);
                    x.cert2_steps = reinterpret_cast<unsigned long long *>(b->ctl_dev + 88);
                }
            }
            // output specialisation: 1 = every frame uint16 counts + RGBA8, 2 =
            // every frame RGBA8 only, 3 = every frame uint8 counts + RGBA8
            // (none with a histogram), else 0
            bool u16_rgba = !host[g].empty(), rgba_only = !host[g].empty(), u8_rgba = !host[g].empty();
            for (const Frame &F : host[g]) {
                u16_rgba = u16_rgba && F.counts && F.count_type == JL_COUNT_U16 && F.rgba && !F.hist_bins;
                rgba_only = rgba_only && !F.counts && F.rgba && !F.hist_bins;
                u8_rgba = u8_rgba && F.counts && F.count_type == JL_COUNT_U8 && F.rgba && !F.hist_bins;
            }
            x.out_mode = u16_rgba ? 1 : rgba_only ? 2 : u8_rgba ? 3 : 0;
            memcpy(x.palette, pal, 1024);
            return x;
        };
        const int sms = device_sm_count();
        if (sms <= 0) { rc = fail(JL_EUNSUPPORTED, "no CUDA device"); break; }
        // Tuned plan: time candidate kernels on the plan's own frames (each run
        // once to warm up, then twice), keep the fastest.  Outputs written by
        // these runs are overwritten by every launch of the plan.
        if (b->tuned[0] || b->tuned[1]) {
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            e = cudaEventCreate(&t0);
            if (e == cudaSuccess)
                e = cudaEventCreate(&t1);
            for (int g = 0; g < 2 && e == cudaSuccess && rc == JL_OK; ++g)
                if (b->n_group[g])
                    e = launch_coords(b->frames_dev[g], nullptr, b->n_group[g], b->s0);
            for (int g = 0; g < 2 && e == cudaSuccess && rc == JL_OK; ++g) {
                if (!b->tuned[g] || !b->n_group[g])
                    continue;
                std::vector<Variant> cand;
                cand.push_back(b->variant[g]);
                if (b->tile_dev[g]) {
                    cand.push_back(Variant{0, 0, 256, 0});
                    if (g == 0) {
                        cand.push_back(Variant{0, 16, 256, 0});
                        cand.push_back(Variant{0, 8, 256, 0});
                    }
                }
                cand.push_back(default_variant(g, 0));
                if (g == 1) {
                    cand.push_back(Variant{2, 4, 256, 0});
                    cand.push_back(Variant{4, 4, 128, 0});
                    cand.push_back(Variant{2, 4, 128, 0});
                    cand.push_back(Variant{4, 4, 256, 0});
                }
                float best_ms = 0.f;
                int best = -1;
                for (size_t ci = 0; ci < cand.size() && e == cudaSuccess; ++ci) {
                    const Variant &v = cand[ci];
                    if (v.ppt == 0 && !b->tile_dev[g])
                        continue;
                    bool seen = false;
                    for (size_t cj = 0; cj < ci; ++cj)
                        seen = seen || (cand[cj].ppt == v.ppt && cand[cj].unroll == v.unroll &&
                                        cand[cj].threads == v.threads);
                    if (seen)
                        continue;
                    const EscapeArgs x = make_args(g, v);
                    float ms = 0.f;
                    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                        e = cudaMemsetAsync(b->ctl_dev, 0, 96, b->s0);
                        if (e == cudaSuccess)
                            e = cudaEventRecord(t0, b->s0);
                        if (e == cudaSuccess)
                            e = launch_escape(x, g, v, sms, b->s0);
                        if (e == cudaSuccess)
                            e = cudaEventRecord(t1, b->s0);
                        if (e == cudaSuccess)
                            e = cudaEventSynchronize(t1);
                        float one = 0.f;
                        if (e == cudaSuccess)
                            e = cudaEventElapsedTime(&one, t0, t1);
                        if (r > 0)
                            ms += one;
                    }
                    // a later candidate must win by more than 1 % (run-to-run noise)
                    if (e == cudaSuccess && (best < 0 || ms < best_ms * 0.99f)) {
                        best = (int)ci;
                        best_ms = ms;
                    }
                }
                if (e == cudaSuccess && best >= 0)
                    b->variant[g] = cand[(size_t)best];
            }
            if (t0)
                cudaEventDestroy(t0);
            if (t1)
                cudaEventDestroy(t1);
            if (e != cudaSuccess) { rc = cuda_fail(e, "plan tuning"); break; }
        }
        for (int g = 0; g < 2; ++g)
            args[g] = make_args(g, b->variant[g]);
        e = cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamBeginCapture"); break; }
        cudaError_t ce = cudaMemsetAsync(b->ctl_dev, 0, 96, b->s0);
        // region covering: coordinate tables of every frame, each launch
        for (int g = 0; g < 2 && ce == cudaSuccess; ++g)
            if (b->n_group[g])
                ce = launch_coords(b->frames_dev[g], nullptr, b->n_group[g], b->s0);
        for (int g = 0; g < 2 && ce == cudaSuccess && any_hist; ++g)
            if (b->n_group[g])
                ce = launch_hist_zero(b->frames_dev[g], b->n_group[g], b->s0);
        b->cert_used = b->n_group[1] && args[1].cert_list && b->variant[1].ppt > 0 && args[1].tile_frame;
        b->cert2_used = b->cert_used && args[1].cert_list2;
        // one group's kernels on stream s, with its timing events when asked for
        auto group = [&](int g, cudaStream_t s) -> cudaError_t {
            cudaEvent_t e0 = b->phases ? b->ph[g ? 2 : 0] : nullptr, e1 = b->phases ? b->ph[g ? 4 : 1] : nullptr;
            cudaEvent_t mid = (b->phases && g) ? b->ph[3] : nullptr, mid2 = (b->phases && g) ? b->ph[5] : nullptr;
            cudaError_t r = e0 ? cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal) : cudaSuccess;
            if (r == cudaSuccess)
                r = launch_escape(args[g], g, b->variant[g], sms, s, mid, mid2, g ? b->certs_done : nullptr);
            if (r == cudaSuccess && e1)
                r = cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
            return r;
        };
        const bool both = b->n_group[0] && b->n_group[1];
        if (ce == cudaSuccess && both) {
            ce = cudaEventRecord(b->fork, b->s0);
            if (ce == cudaSuccess)
                ce = cudaStreamWaitEvent(b->s1, b->fork, 0);
            if (ce == cudaSuccess)
                ce = group(1, b->s1);
            if (ce == cudaSuccess)
                ce = cudaEventRecord(b->join, b->s1);
            // With the certified passes the binary64 group starts with two
            // binary32-pipe kernels, then its binary64 kernel leaves the
            // binary32 pipe idle: the binary32 frames run beside the latter.
            if (ce == cudaSuccess && b->cert_used)
                ce = cudaStreamWaitEvent(b->s0, b->certs_done, 0);
            if (ce == cudaSuccess)
                ce = group(0, b->s0);
            if (ce == cudaSuccess)
                ce = cudaStreamWaitEvent(b->s0, b->join, 0);
        } else if (ce == cudaSuccess) {
            ce = group(b->n_group[0] ? 0 : 1, b->s0);
        }
        for (int g = 0; g < 2 && ce == cudaSuccess && any_hist; ++g)
            if (b->n_group[g])
                ce = launch_hist_finalize(b->frames_dev[g], nullptr, b->n_group[g], b->s0);
        e = cudaStreamEndCapture(b->s0, &b->graph);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "graph capture"); break; }
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamEndCapture"); break; }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGraphInstantiate"); break; }
    } while (0);
    if (rc != JL_OK) {
        destroy_plan(b);
        return rc;
    }
    *out = b;
    return JL_OK;
}

int jl_batch_variant(const jl_batch *b, int32_t precision, int32_t *ppt, int32_t *unroll, int32_t *threads)
{
    if (!b || (precision != JL_FP32 && precision != JL_FP64))
        return fail(JL_EINVAL, "invalid arguments");
    const Variant &v = b->variant[precision];
    if (ppt)
        *ppt = v.ppt;
    if (unroll)
        *unroll = v.unroll;
    if (threads)
        *threads = v.threads;
    return JL_OK;
}

int jl_batch_launch(jl_batch *b, void *stream)
{
    if (!b || !b->exec)
        return fail(JL_EINVAL, "invalid batch plan");
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphLaunch");
    return JL_OK;
}

int jl_batch_status(jl_batch *b, void *stream, int32_t *status_out)
{
    if (!b || !status_out)
        return fail(JL_EINVAL, "invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b->ctl_dev + 16, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading batch status");
    *status_out = v;
    return JL_OK;
}

int jl_batch_cert_stats(jl_batch *b, void *stream, int64_t *out)
{
    if (!b || !out)
        return fail(JL_EINVAL, "invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(v, b->ctl_dev + 32, 64, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the certified passes' counters");
    out[0] = (int64_t)v[0];
    out[1] = (int64_t)(b->cert2_used ? v[3] : v[0]);
    out[2] = (int64_t)v[5];
    out[3] = (int64_t)v[2];
    out[4] = (int64_t)v[6];
    out[5] = (int64_t)v[7];
    return JL_OK;
}

int jl_batch_phase_ms(const jl_batch *b, float *ms_out)
{
    if (!b || !ms_out)
        return fail(JL_EINVAL, "invalid arguments");
    if (!b->phases)
        return fail(JL_EINVAL, "the plan was created without phase events (opts.variant_flags bit 3)");
    for (int k = 0; k < 4; ++k)
        ms_out[k] = -1.f;
    cudaError_t e = cudaSuccess;
    if (b->n_group[0])
        e = cudaEventElapsedTime(&ms_out[0], b->ph[0], b->ph[1]);
    if (e == cudaSuccess && b->n_group[1]) {
        if (b->cert_used) {
            e = cudaEventElapsedTime(&ms_out[1], b->ph[2], b->ph[3]);
            if (e == cudaSuccess && b->cert2_used)
                e = cudaEventElapsedTime(&ms_out[2], b->ph[3], b->ph[5]);
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms_out[3], b->ph[5], b->ph[4]);
        } else {
            e = cudaEventElapsedTime(&ms_out[3], b->ph[2], b->ph[4]);
        }
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "reading phase events");
    return JL_OK;
}

int jl_batch_precisions(const jl_batch *b, int32_t *out, int32_t cap)
{
    if (!b)
        return fail(-1, "invalid batch plan");
    for (int i = 0; i < b->n && i < cap && out; ++i)
        out[i] = b->prec[i];
    return b->n;
}

int jl_batch_pixels(const jl_batch *b, int64_t *fp32_pixels, int64_t *fp64_pixels)
{
    if (!b)
        return fail(JL_EINVAL, "invalid batch plan");
    if (fp32_pixels)
        *fp32_pixels = b->pixels[0];
    if (fp64_pixels)
        *fp64_pixels = b->pixels[1];
    return JL_OK;
}

void jl_batch_destroy(jl_batch *b) { destroy_plan(b); }

int jl_render_batch(const jl_frame *frames, int32_t n, void *counts_base, uint8_t *rgba_base, float *hist_base,
                    const uint8_t *palette, void *stream)
{
    jl_batch *b = nullptr;
    int rc = jl_batch_create(frames, n, counts_base, rgba_base, hist_base, palette, nullptr, &b);
    if (rc != JL_OK)
        return rc;
    rc = jl_batch_launch(b, stream);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (rc == JL_OK && e != cudaSuccess)
        rc = cuda_fail(e, "cudaStreamSynchronize");
    int32_t st = 0;
    if (rc == JL_OK && jl_batch_status(b, stream, &st) == JL_OK && st != 0)
        rc = fail(st, "batch stopped early (status " + std::to_string(st) + ")");
    destroy_plan(b);
    return rc;
}

}  // extern "C"
