// Escape-time kernels for sm_103a (paper Sec. 2: region covering and the
// escape-time iteration of Z <- Z^2 + C; Sec. 3: Mandelbrot mode, deep zoom).
//
// Design (B300-first, not the paper's one-thread-per-pixel kernel):
//  * Coordinates.  x_i and y_j depend on one index each, so they are computed
//    once per frame into tables (W + H values) by `coords_kernel`, in binary64
//    without FMA, then rounded once to the working type.  This keeps binary64
//    work (a narrow pipe on this part) out of the per-pixel path.
//  * Persistent warps with lane refill.  Each warp pulls row segments
//    ("chunks") from a global atomic counter and keeps PPT independent pixels
//    per lane in flight (ILP).  A lane whose pixel finishes stores its result
//    and takes the next pixel of the warp's chunk at the next service point,
//    so escaped lanes do not idle while their neighbours keep iterating.
//  * Blocks of U steps.  Between service points every slot runs U steps with
//    no branch.  The escape test stays exact:
//      - binary32: the value r_u = x2 + y2 of every step is kept in registers;
//        because escape is monotone for the pixels that take this path (see
//        `monotone_*` below) the slot escaped in the block iff r_{U-1} fails,
//        and the count is n + #{u : r_u <= 4};
//      - binary64: r is not formed in binary64.  A binary32 estimate built
//        from the high words of x2 and y2 decides the test whenever it is
//        outside a +-2^-16 relative band around 4; a block in which any live
//        slot fell inside the band is replayed with exact binary64 tests.
//    Pixels for which monotonicity is not proven (|C| within 2^-12 of 2) and
//    tails shorter than U steps are iterated one exact step at a time.
//  * Binary64 frames first go through two certified passes (`cert_kernel`,
//    `cert2_kernel`): a binary32, then a float-pair, orbit with a rigorous
//    bound on its distance to the binary64 orbit decides each binary64 test
//    it can; only the pixels with a test neither settles are iterated in
//    binary64 (the lane-refill kernel over their list).  The counts are the
//    binary64 counts either way.
//  * Every arithmetic operation of an orbit whose counts are reported is an
//    explicit round-to-nearest intrinsic (__fmul_rn, __fadd_rn, __dmul_rn,
//    ...), which the compiler never contracts into an FMA; the library is
//    also built with -fmad=false.  The certified passes' approximate orbits
//    use FMA deliberately (their bound accounts for every rounding).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <math.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "jl_common.cuh"
#include "jl_internal.h"

namespace jl {

static constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Region covering (Sec. 2): coordinate tables.
// Block b handles frame b / 2, axis b % 2 (0: x over W, 1: y over H).
// ---------------------------------------------------------------------------
struct CoordArgs {
    const Frame *frames;
    int32_t n_frames;
    Frame single;
};

__global__ void coords_kernel(const __grid_constant__ CoordArgs a)
{
    const Frame *frames = a.frames ? a.frames : &a.single;
    const int f = blockIdx.x >> 1;
    const int axis = blockIdx.x & 1;
    if (f >= a.n_frames)
        return;
    const Frame &F = frames[f];
    const int n = axis ? F.H : F.W;
    const double lo = axis ? F.ymin : F.xmin;
    const double d = axis ? F.dy : F.dx;
    void *out = const_cast<void *>(axis ? F.ys : F.xs);
    // binary64 frames: also the binary32 roundings for the certified pass and
    // the remainders (exact in binary64) rounded to binary32 for the double-float pass
    float *out32 = F.precision == JL_FP64 ? const_cast<float *>(axis ? F.ys32 : F.xs32) : nullptr;
    float *out32lo = F.precision == JL_FP64 ? const_cast<float *>(axis ? F.ys32lo : F.xs32lo) : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // lo + (i + 0.5) * d, binary64, no contraction.
        double t = __dadd_rn((double)i, 0.5);
        double v = __dadd_rn(lo, __dmul_rn(t, d));
        if (F.precision == JL_FP64) {
            static_cast<double *>(out)[i] = v;
            if (out32) {
                const float h = __double2float_rn(v);
                out32[i] = h;
                if (out32lo)
                    out32lo[i] = __double2float_rn(__dsub_rn(v, (double)h));
            }
        } else {
            static_cast<float *>(out)[i] = __double2float_rn(v);
        }
    }
}

// ---------------------------------------------------------------------------
// Histogram finalisation: bins (uint32, in place) -> binary32 fractions.
// ---------------------------------------------------------------------------
struct HistArgs {
    const Frame *frames;
    int32_t n_frames;
    Frame single;
};

__global__ void hist_finalize_kernel(const __grid_constant__ HistArgs a)
{
    const Frame *frames = a.frames ? a.frames : &a.single;
    for (int f = blockIdx.x; f < a.n_frames; f += gridDim.x) {
        const Frame &F = frames[f];
        if (!F.hist_bins)
            continue;
        const double npix = (double)F.W * (double)F.H;
        for (int b = threadIdx.x; b <= F.max_iter; b += blockDim.x) {
            uint32_t c = F.hist_bins[b];
            float v = __double2float_rn(__ddiv_rn((double)c, npix));
            reinterpret_cast<float *>(F.hist_bins)[b] = v;
        }
    }
}

// Zero the uint32 bins of every frame that has a histogram (batch launches).
__global__ void hist_zero_kernel(const __grid_constant__ HistArgs a)
{
    const Frame *frames = a.frames ? a.frames : &a.single;
    for (int f = blockIdx.x; f < a.n_frames; f += gridDim.x) {
        const Frame &F = frames[f];
        if (!F.hist_bins)
            continue;
        for (int b = threadIdx.x; b <= F.max_iter; b += blockDim.x)
            F.hist_bins[b] = 0u;
    }
}

__global__ void dbl2_kernel(const double *in, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = dbl2(in[i]);
}

cudaError_t launch_dbl2(const double *in, double *out, int n, cudaStream_t st)
{
    dbl2_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact single-step iteration (used for tails, unproven-monotone pixels and
// nothing else).  Returns the count given that tests 0..n0-1 have passed and
// (x, y) is Z_{n0}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int exact_from(float x, float y, float cr, float ci, int n0, int max_iter)
{
    for (int n = n0; n < max_iter; ++n) {
        float x2 = __fmul_rn(x, x);
        float y2 = __fmul_rn(y, y);
        if (__fadd_rn(x2, y2) > 4.0f)
            return n;
        float t = __fadd_rn(x, x);
        t = __fmul_rn(t, y);
        y = __fadd_rn(t, ci);
        x = __fadd_rn(__fsub_rn(x2, y2), cr);
    }
    return max_iter;
}

__device__ __forceinline__ int exact_from(double x, double y, double cr, double ci, int n0, int max_iter)
{
    for (int n = n0; n < max_iter; ++n) {
        double x2 = __dmul_rn(x, x);
        double y2 = __dmul_rn(y, y);
        if (__dadd_rn(x2, y2) > 4.0)
            return n;
        double t = dbl2(x);
        t = __dmul_rn(t, y);
        y = __dadd_rn(t, ci);
        x = __dadd_rn(__dsub_rn(x2, y2), cr);
    }
    return max_iter;
}

// Monotone escape.  If |C| <= 2 - 2^-12 then, in binary32 or binary64
// arithmetic with round-to-nearest, a failed test (x2 + y2 > 4) at step m
// implies |Z_{m+1}| >= 2 + 2^-13 and the modulus keeps growing until it
// overflows to inf/NaN, so every later test also fails (NaN fails "<= 4").
// For Mandelbrot pixels with |C| >= 2 + 2^-12, Z_1 = C fails the test and the
// same growth holds from there on.  Pixels with |C| in between are iterated
// exactly one step at a time.  The band is tested here with margin so that
// rounding in |C|^2 cannot hide a pixel that belongs to it.
__device__ __forceinline__ bool in_unsafe_band(double cr, double ci)
{
    double m = __dadd_rn(__dmul_rn(cr, cr), __dmul_rn(ci, ci));
    return m > 3.99 && m < 4.01;
}
__device__ __forceinline__ bool in_unsafe_band(float cr, float ci)
{
    float m = __fadd_rn(__fmul_rn(cr, cr), __fmul_rn(ci, ci));
    return m > 3.99f && m < 4.01f;
}

// ---------------------------------------------------------------------------
// The persistent escape kernel.
// ---------------------------------------------------------------------------
// C of a Julia frame in the working type (binary32 value rounded on the host).
template <typename T>
struct WorkT;
template <>
struct WorkT<float> {
    static __device__ __forceinline__ float cr(const Frame &F) { return F.cr32; }
    static __device__ __forceinline__ float ci(const Frame &F) { return F.ci32; }
};
template <>
struct WorkT<double> {
    static __device__ __forceinline__ double cr(const Frame &F) { return F.cr; }
    static __device__ __forceinline__ double ci(const Frame &F) { return F.ci; }
};

// One pixel's state in the binary64 kernel's end-of-launch packing area.
struct TailSlot {
    double x, y, cr, ci;
    int32_t rem, fid, pix, pad;
};

// Dynamic shared memory of the lane-refill kernel: the palette, the
// histogram of a single frame (hist_words, 0 for none), and for binary64 with
// several slots per lane the warps' packing areas.
static size_t refill_smem_bytes(bool dbl, int ppt, int threads, size_t hist_words)
{
    size_t words = ((256 + hist_words + 1) & ~(size_t)1);
    size_t bytes = words * sizeof(uint32_t);
    if (dbl && ppt > 1)
        bytes += (size_t)(threads / 32) * (size_t)ppt * 32 * sizeof(TailSlot);
    return bytes;
}

// LIST (binary64): the pixels are the entries of the certified pass's list
// (a.cert_list, *a.cert_count of them) instead of the frames' row chunks.
template <typename T, int PPT, int U, bool BATCH, bool LIST>
__global__ void __launch_bounds__(256) escape_kernel(const __grid_constant__ EscapeArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t *pal = smem;
    uint32_t *hbins = smem + 256;
    // binary64 with several slots: each warp's area for packing its pixels at
    // the end of the launch, after the palette and the histogram (8-aligned)
    const int nb_words = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    TailSlot *tail_slots = reinterpret_cast<TailSlot *>(smem + ((256 + nb_words + 1) & ~1));

    const int lane = threadIdx.x & 31;
    const unsigned lane_bit = 1u << lane;
    const unsigned lt_mask = lane_bit - 1u;

    // Frame f of the launch: the table in global memory for batches, the
    // launch parameters for single frames.
    auto FR = [&](int f) -> const Frame & {
        if constexpr (BATCH)
            return a.frames[f];
        else
            return a.single;
    };

    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    const long long t_start = clock64();

    // ---- warp work queue (warp-uniform state) ----
    // A chunk is rows [q_j0, q_j0 + k) x columns [q_x0, q_x0 + q_span) of frame
    // q_f, its pixels numbered o = 0 .. q_end-1 row-major; row offset of o is
    // (o * q_magic) >> 20 (exact for o < 1024 <= 2^20 / span, see make_frame).
    int q_f = 0, q_j0 = 0, q_x0 = 0, q_span = 1, q_pos = 0, q_end = 0, q_W = 0, q_max = 0, q_mode = 0;
    int q_safe = 1;
    uint32_t q_magic = 0;
    T q_cr = T(0), q_ci = T(0);
    const T *q_xs = nullptr;
    const T *q_ys = nullptr;
    bool q_done = false;
    unsigned long long next_c = 0;  // valid in lane 0: prefetched chunk id
    if (lane == 0)
        next_c = atomicAdd(a.chunk_counter, 1ull);
    // LIST: entries of the list and its 32-entry pieces (the chunks here)
    long long list_n = 0, q_l0 = 0;
    if constexpr (LIST) {
        list_n = (long long)*a.cert_count;
        if (list_n > a.cert_cap)
            list_n = a.cert_cap;
    }
    const long long total_chunks = LIST ? (list_n + 31) >> 5 : a.total_chunks;

    auto advance = [&]() -> bool {
        if (q_done)
            return false;
        unsigned long long c = __shfl_sync(FULL, next_c, 0);
        bool over_budget = false;
        if (a.cycle_budget > 0 && (clock64() - t_start) > a.cycle_budget)
            over_budget = true;
        over_budget = __any_sync(FULL, over_budget);
        if ((long long)c >= total_chunks || over_budget) {
            if (over_budget && lane == 0 && a.status && (long long)c < total_chunks)
                atomicExch(a.status, (int)JL_ETIMEOUT);
            q_done = true;
            return false;
        }
        if (lane == 0)
            next_c = atomicAdd(a.chunk_counter, 1ull);
        if constexpr (LIST) {
            q_l0 = (long long)c << 5;
            q_pos = 0;
            q_end = (int)min(32ll, list_n - q_l0);
            return true;
        }
        int f = 0;
        if constexpr (BATCH)
            f = a.chunk_frame[c];
        const Frame &F = FR(f);
        const int lc = (int)((long long)c - F.chunk_begin);
        q_f = f;
        if (F.rows_per_chunk > 1) {
            q_j0 = lc * F.rows_per_chunk;
            q_x0 = 0;
            q_span = F.W;
            q_end = min(F.rows_per_chunk, F.H - q_j0) * F.W;
            q_magic = F.span_magic;
        } else {
            const int row = lc / F.chunks_per_row;
            const int seg = lc - row * F.chunks_per_row;
            q_j0 = row;
            q_x0 = seg * F.chunk_len;
            q_span = min(F.chunk_len, F.W - q_x0);
            q_end = q_span;
            q_magic = 0;
        }
        q_pos = 0;
        q_W = F.W;
        q_max = F.max_iter;
        q_mode = F.mode;
        q_safe = F.safe;
        q_cr = WorkT<T>::cr(F);
        q_ci = WorkT<T>::ci(F);
        q_xs = static_cast<const T *>(F.xs);
        q_ys = static_cast<const T *>(F.ys);
        return true;
    };

    // ---- slot state ----
    // rem >= 0: live, rem = max_iter - n (tests still allowed);
    // rem < 0 : finished early, count = -1 - rem;  fid < 0: empty.
    T x[PPT], y[PPT], cr[PPT], ci[PPT];
    int rem[PPT], fid[PPT], pix[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        x[k] = y[k] = cr[k] = ci[k] = T(0);
        rem[k] = 0x3fffffff;
        fid[k] = -1;
        pix[k] = 0;
    }

    // Store one finished pixel (count, colour, histogram bin).  Called by the
    // lanes that finished a pixel in this slot (a divergent region).
    auto finish = [&](int f, int p, int count) {
        const Frame &F = FR(f);
        if (F.counts) {
            if (F.count_type == JL_COUNT_U8)
                F.counts[p] = (uint8_t)count;
            else
                reinterpret_cast<uint16_t *>(F.counts)[p] = (uint16_t)count;
        }
        if (F.rgba)
            F.rgba[p] = pal[colour_index((uint32_t)count, (uint32_t)F.max_iter, F.colour_magic)];
        if (LIST && a.list_iters) {
            const unsigned act = __activemask();
            const unsigned tot = __reduce_add_sync(act, (unsigned)count);
            if ((act & lt_mask) == 0)
                atomicAdd(a.list_iters, (unsigned long long)tot);
        }
        if (F.hist_bins) {
            if (!BATCH && a.hist_smem) {
                atomicAdd(&hbins[count], 1u);
            } else {
                // one atomic per distinct (frame, count) among the active lanes
                const unsigned act = __activemask();
                const unsigned long long key = ((unsigned long long)(unsigned)f << 32) | (unsigned)count;
                const unsigned grp = __match_any_sync(act, key);
                if ((grp & lt_mask) == 0)
                    atomicAdd(&F.hist_bins[count], (unsigned)__popc(grp));
            }
        }
    };

    // Assign new pixels to slot k for the lanes in `want`.
    auto refill = [&](int k, unsigned want) {
        unsigned remaining = want;
        while (remaining) {
            if (q_pos >= q_end) {
                if (!advance())
                    break;
                continue;
            }
            const int avail = q_end - q_pos;
            const int take = min(avail, __popc(remaining));
            const bool mine = (remaining & lane_bit) != 0;
            const int rank = __popc(remaining & lt_mask);
            const bool got = mine && rank < take;
            if (LIST && got) {
                // list entry (frame << 32) | (row << 16) | column, taken from the
                // list's end: the double-float pass appends a pixel when its test
                // fails, so the longest-lived pixels come last and start first here
                const uint64_t ent = a.cert_list[list_n - 1 - (q_l0 + q_pos + rank)];
                const int f = (int)(ent >> 32);
                const int j = (int)((ent >> 16) & 0xffffu);
                const int i = (int)(ent & 0xffffu);
                const Frame &F = FR(f);
                const T xv = static_cast<const T *>(F.xs)[i];
                const T yv = static_cast<const T *>(F.ys)[j];
                fid[k] = f;
                pix[k] = j * F.W + i;
                rem[k] = F.max_iter;
                bool unsafe;
                if (F.mode == JL_JULIA) {
                    x[k] = xv;
                    y[k] = yv;
                    cr[k] = WorkT<T>::cr(F);
                    ci[k] = WorkT<T>::ci(F);
                    unsafe = !F.safe;
                } else {
                    x[k] = T(0);
                    y[k] = T(0);
                    cr[k] = xv;
                    ci[k] = yv;
                    unsafe = in_unsafe_band(xv, yv);
                }
                if (unsafe || F.max_iter < U) {
                    const int c = exact_from(x[k], y[k], cr[k], ci[k], 0, F.max_iter);
                    rem[k] = -1 - c;
                }
            } else if (got) {
                const int o = q_pos + rank;
                const int jj = (int)(((uint32_t)o * q_magic) >> 20);
                const int i = q_x0 + o - jj * q_span;
                const int j = q_j0 + jj;
                const T xv = q_xs[i];
                const T yv = q_ys[j];
                fid[k] = q_f;
                pix[k] = j * q_W + i;
                rem[k] = q_max;
                bool unsafe;
                if (q_mode == JL_JULIA) {
                    x[k] = xv;
                    y[k] = yv;
                    cr[k] = q_cr;
                    ci[k] = q_ci;
                    unsafe = !q_safe;
                } else {
                    x[k] = T(0);
                    y[k] = T(0);
                    cr[k] = xv;
                    ci[k] = yv;
                    unsafe = in_unsafe_band(xv, yv);
                }
                if (unsafe || q_max < U) {
                    const int c = exact_from(x[k], y[k], cr[k], ci[k], 0, q_max);
                    rem[k] = -1 - c;
                }
            }
            remaining &= ~__ballot_sync(FULL, got);
            q_pos += take;
        }
    };

    // Initial fill.
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        refill(k, FULL);

    // Per-slot "needs service" flags computed after each block.
    bool need[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        need[k] = false;

    float rk[PPT][U];   // binary32 path: r_u of the last block
    int cnt[PPT];       // binary64 path: passed tests in the last block

    while (true) {
        // ---------------- service ----------------
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (__any_sync(FULL, need[k])) {
                if (need[k]) {
                    int count;
                    const int f = fid[k];
                    const int mi = FR(f).max_iter;
                    if (rem[k] < 0) {
                        count = -1 - rem[k];
                    } else if (rem[k] < U) {
                        // tail shorter than a block: exact steps from n = mi - rem
                        count = exact_from(x[k], y[k], cr[k], ci[k], mi - rem[k], mi);
                    } else {
                        // escaped inside the last block (tests n .. n+U-1, n = mi - rem)
                        int passed;
                        if constexpr (sizeof(T) == 4) {
                            passed = 0;
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                passed += (rk[k][u] <= 4.0f) ? 1 : 0;
                        } else {
                            passed = cnt[k];
                        }
                        count = mi - rem[k] + passed;
                    }
                    finish(f, pix[k], count);
                    fid[k] = -1;
                    rem[k] = 0x3fffffff;
                    x[k] = y[k] = cr[k] = ci[k] = T(0);
                }
                const unsigned want = __ballot_sync(FULL, need[k]);
                if (!q_done)
                    refill(k, want);
            }
        }

        bool live = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k)
            live |= (fid[k] >= 0);
        if (!__any_sync(FULL, live))
            break;

        // ---------------- block of U steps ----------------
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    float xx = (float)x[k], yy = (float)y[k];
                    float x2 = __fmul_rn(xx, xx);
                    float y2 = __fmul_rn(yy, yy);
                    rk[k][u] = __fadd_rn(x2, y2);
                    float t = __fadd_rn(xx, xx);
                    t = __fmul_rn(t, yy);
                    y[k] = (T)__fadd_rn(t, (float)ci[k]);
                    x[k] = (T)__fadd_rn(__fsub_rn(x2, y2), (float)cr[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const bool live_k = rem[k] >= 0 && fid[k] >= 0;
                const bool esc = !(rk[k][U - 1] <= 4.0f);
                if (live_k && !esc)
                    rem[k] -= U;
                need[k] = (fid[k] >= 0) && (!live_k || esc || rem[k] < U);
            }
        } else {
            // Binary64 block; GUARD: only the first nslot slots (the others are
            // empty in every lane of the warp).
            auto block64 = [&](auto guard, int nslot) {
                constexpr bool GUARD = decltype(guard)::value;
                double sx[PPT], sy[PPT];
                bool amb = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    sx[k] = (double)x[k];
                    sy[k] = (double)y[k];
                    cnt[k] = 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (GUARD && k >= nslot)
                            continue;
                        double xx = (double)x[k], yy = (double)y[k];
                        double x2 = __dmul_rn(xx, xx);
                        double y2 = __dmul_rn(yy, yy);
                        float r32 = __fadd_rn(hi_estimate(x2), hi_estimate(y2));
                        cnt[k] += (r32 < 3.9999847412109375f) ? 1 : 0;
                        amb |= (rem[k] >= 0) & (r32 >= 3.9999847412109375f) & (r32 <= 4.0000152587890625f);
                        double t = dbl2(xx);
                        t = __dmul_rn(t, yy);
                        y[k] = (T)__dadd_rn(t, (double)ci[k]);
                        x[k] = (T)__dadd_rn(__dsub_rn(x2, y2), (double)cr[k]);
                    }
                }
                if (__any_sync(FULL, amb)) {
                    // replay the block with exact binary64 tests
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        x[k] = (T)sx[k];
                        y[k] = (T)sy[k];
                        cnt[k] = 0;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            if (GUARD && k >= nslot)
                                continue;
                            double xx = (double)x[k], yy = (double)y[k];
                            double x2 = __dmul_rn(xx, xx);
                            double y2 = __dmul_rn(yy, yy);
                            cnt[k] += (__dadd_rn(x2, y2) <= 4.0) ? 1 : 0;
                            double t = dbl2(xx);
                            t = __dmul_rn(t, yy);
                            y[k] = (T)__dadd_rn(t, (double)ci[k]);
                            x[k] = (T)__dadd_rn(__dsub_rn(x2, y2), (double)cr[k]);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const bool live_k = rem[k] >= 0 && fid[k] >= 0;
                    const bool esc = cnt[k] < U;
                    if (live_k && !esc)
                        rem[k] -= U;
                    need[k] = (fid[k] >= 0) && (!live_k || esc || rem[k] < U);
                }
            };
            int nslot = PPT;
            if (PPT > 1 && q_done) {
                // No pixels are left to take: the warp's pixels are packed
                // into its lowest slots across all lanes (through shared
                // memory), and the slots no lane then uses are not computed (a
                // binary64 warp instruction costs the narrow pipe the same
                // whatever its lanes hold).
                unsigned bal[PPT];
                int base[PPT];
                int tot = 0;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    bal[k] = __ballot_sync(FULL, fid[k] >= 0);
                    base[k] = tot;
                    tot += __popc(bal[k]);
                }
                nslot = (tot + 31) >> 5;
                if (nslot < PPT) {
                    TailSlot *ts = tail_slots + (threadIdx.x >> 5) * (PPT * 32);
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (fid[k] >= 0) {
                            TailSlot &d = ts[base[k] + __popc(bal[k] & lt_mask)];
                            d.x = x[k];
                            d.y = y[k];
                            d.cr = cr[k];
                            d.ci = ci[k];
                            d.rem = rem[k];
                            d.fid = fid[k];
                            d.pix = pix[k];
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const int g = k * 32 + lane;
                        if (g < tot) {
                            const TailSlot &d = ts[g];
                            x[k] = d.x;
                            y[k] = d.y;
                            cr[k] = d.cr;
                            ci[k] = d.ci;
                            rem[k] = d.rem;
                            fid[k] = d.fid;
                            pix[k] = d.pix;
                        } else {
                            x[k] = y[k] = cr[k] = ci[k] = T(0);
                            rem[k] = 0x3fffffff;
                            fid[k] = -1;
                        }
                    }
                    __syncwarp();
                }
            }
            if (nslot == PPT)
                block64(std::integral_constant<bool, false>(), PPT);
            else
                block64(std::integral_constant<bool, true>(), nslot);
        }
    }

    if (nb) {
        __syncthreads();
        uint32_t *gb = a.single.hist_bins;
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            uint32_t v = hbins[t];
            if (v)
                atomicAdd(&gb[t], v);
        }
    }
}


// Escape count of one pixel in blocks of 4 steps with one branch per block.
// When escape is monotone (`mono`, see in_unsafe_band) the block keeps the
// squares of its four steps, forms only the last test value r = x2 + y2 on
// the way and, once that one fails, the count is the number of passed tests
// (the first three r formed on the exit path from the kept squares: the same
// roundings); otherwise every step is tested exactly.
template <typename T>
__device__ __forceinline__ int escape_blocked(T x, T y, T cr, T ci, int max_iter, bool mono)
{
    if (!mono)
        return exact_from(x, y, cr, ci, 0, max_iter);
    int n = 0;
    for (; n + 4 <= max_iter; n += 4) {
        T x2s[4], y2s[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            T t;
            if constexpr (sizeof(T) == 4) {
                x2s[u] = __fmul_rn(x, x);
                y2s[u] = __fmul_rn(y, y);
                t = __fmul_rn(__fadd_rn(x, x), y);
                y = __fadd_rn(t, ci);
                x = __fadd_rn(__fsub_rn(x2s[u], y2s[u]), cr);
            } else {
                x2s[u] = __dmul_rn(x, x);
                y2s[u] = __dmul_rn(y, y);
                t = __dmul_rn(dbl2(x), y);
                y = __dadd_rn(t, ci);
                x = __dadd_rn(__dsub_rn(x2s[u], y2s[u]), cr);
            }
        }
        T r3;
        if constexpr (sizeof(T) == 4)
            r3 = __fadd_rn(x2s[3], y2s[3]);
        else
            r3 = __dadd_rn(x2s[3], y2s[3]);
        if (!(r3 <= T(4))) {
            int passed = 0;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                T r;
                if constexpr (sizeof(T) == 4)
                    r = __fadd_rn(x2s[u], y2s[u]);
                else
                    r = __dadd_rn(x2s[u], y2s[u]);
                passed += (r <= T(4)) ? 1 : 0;
            }
            return n + passed;
        }
    }
    // tail shorter than a block: Z_n is (x, y)
    return exact_from(x, y, cr, ci, n, max_iter);
}

// ---------------------------------------------------------------------------
// Compacting tile kernel (binary32).
//
// The static kernel's two losses on low-count frames are per-pixel
// instructions and warp divergence: a warp runs as long as the slowest of its
// 32 pixels while finished lanes idle.  Here each warp walks the same 8 x 4
// patches as the static kernel, but a patch whose live lanes have dropped to
// `T` or fewer (checked after the first 16 steps and after every super-block)
// parks them: the live lanes write their
// state (Z, C, n, pixel, frame) to a ring of 64 entries owned by the warp in
// shared memory, and the warp moves on.  Once 32 parked pixels have
// accumulated the warp resumes them together as one full batch (which may park
// its own stragglers again).  At the end the warp merges what is left into its
// last batches.  Parked pixels continue from exactly where they stopped, so the
// arithmetic of every pixel is the same sequence of steps as the oracle's.
//
// A patch runs its first 16 steps in blocks of four, then super-blocks of
// four blocks of S2 steps, with the monotone blocked test of `escape_blocked`
// (the count is n + the number of passed tests in the block whose last test
// failed; only that last test value is formed on the way).  A lane that cannot
// run a whole super-block before its limit finishes with `escape_from` (blocks
// of four, then exact single steps).
// ---------------------------------------------------------------------------
static constexpr int kQCap = 64;  // parked pixels per warp (power of two)

struct ParkRing {
    float x[kQCap], y[kQCap], cr[kQCap], ci[kQCap];
    int32_t n[kQCap], f[kQCap];
    uint32_t p[kQCap];
};

// Count of a pixel whose tests 0..n-1 passed, from Z_n = (x, y).
__device__ __forceinline__ int escape_from(float x, float y, float cr, float ci, int n, int max_iter)
{
    for (; n + 4 <= max_iter; n += 4) {
        float r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float x2 = __fmul_rn(x, x);
            const float y2 = __fmul_rn(y, y);
            r[u] = __fadd_rn(x2, y2);
            const float t = __fmul_rn(__fadd_rn(x, x), y);
            y = __fadd_rn(t, ci);
            x = __fadd_rn(__fsub_rn(x2, y2), cr);
        }
        if (!(r[3] <= 4.0f))
            return n + (r[0] <= 4.0f) + (r[1] <= 4.0f) + (r[2] <= 4.0f);
    }
    return exact_from(x, y, cr, ci, n, max_iter);
}

// One binary32 step of Z <- Z^2 + C, returning the test value x^2 + y^2 of Z.
__device__ __forceinline__ float step32(float &x, float &y, float cr, float ci)
{
    const float x2 = __fmul_rn(x, x);
    const float y2 = __fmul_rn(y, y);
    const float r = __fadd_rn(x2, y2);
    const float t = __fmul_rn(__fadd_rn(x, x), y);
    y = __fadd_rn(t, ci);
    x = __fadd_rn(__fsub_rn(x2, y2), cr);
    return r;
}

// Four blocks of S steps each (4 S steps) from Z_n with the monotone blocked
// test.  Returns the count of a pixel whose test failed in one of the blocks,
// else -1 (Z_{n+4S} is then in x, y).  Only the last test value of a block is
// formed on the way; the others (x2 + y2 of the earlier steps) are formed on
// the exit path from the squares kept in registers.
template <int S>
__device__ __forceinline__ int superblock(float &x, float &y, float cr, float ci, int n)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float x2s[S], y2s[S];
#pragma unroll
        for (int u = 0; u < S; ++u) {
            const float x2 = __fmul_rn(x, x);
            const float y2 = __fmul_rn(y, y);
            x2s[u] = x2;
            y2s[u] = y2;
            const float t = __fmul_rn(__fadd_rn(x, x), y);
            y = __fadd_rn(t, ci);
            x = __fadd_rn(__fsub_rn(x2, y2), cr);
        }
        if (!(__fadd_rn(x2s[S - 1], y2s[S - 1]) <= 4.0f)) {
            int passed = 0;
#pragma unroll
            for (int u = 0; u < S - 1; ++u)
                passed += (__fadd_rn(x2s[u], y2s[u]) <= 4.0f) ? 1 : 0;
            return n + S * b + passed;
        }
    }
    return -1;
}

// Output fields of the frame of a tile, held in registers for its patches
// (loads from the frame table could not be hoisted past the output stores).
struct TileOut {
    uint8_t *counts;
    uint32_t *rgba;
    uint32_t *bins;
    uint64_t magic;  // colour reciprocal (40-bit, exact for any limit)
    uint32_t m32;    // floor(2^32 / max_iter) + 1: exact count*255/max_iter for max_iter <= 4096
    int mi;
    bool u8, small;
};

__device__ __forceinline__ uint32_t tile_colour(const TileOut &o, int count)
{
    if (count >= o.mi)
        return 255u;
    return o.small ? __umulhi((uint32_t)count * 255u, o.m32)
                   : (uint32_t)(((uint64_t)((uint32_t)count * 255u) * o.magic) >> 40);
}

template <bool BATCH, int OUT>
__device__ __forceinline__ void store_tile(const EscapeArgs &a, const TileOut &o, const uint32_t *pal,
                                           uint32_t *hbins, int fr, uint32_t p, int count, unsigned lt_mask)
{
    if constexpr (OUT == 1) {
        // uint16 counts and RGBA8, no histogram: no per-frame tests
        reinterpret_cast<uint16_t *>(o.counts)[p] = (uint16_t)count;
        o.rgba[p] = pal[tile_colour(o, count)];
        return;
    }
    if constexpr (OUT == 2) {
        // RGBA8 only
        o.rgba[p] = pal[tile_colour(o, count)];
        return;
    }
    if constexpr (OUT == 3) {
        // uint8 counts and RGBA8, no histogram
        o.counts[p] = (uint8_t)count;
        o.rgba[p] = pal[tile_colour(o, count)];
        return;
    }
    if (o.counts) {
        if (o.u8)
            o.counts[p] = (uint8_t)count;
        else
            reinterpret_cast<uint16_t *>(o.counts)[p] = (uint16_t)count;
    }
    if (o.rgba)
        o.rgba[p] = pal[tile_colour(o, count)];
    if (o.bins) {
        if (!BATCH && a.hist_smem) {
            atomicAdd(&hbins[count], 1u);
        } else {
            const unsigned act = __activemask();
            const unsigned long long key = ((unsigned long long)(unsigned)fr << 32) | (unsigned)count;
            const unsigned grp = __match_any_sync(act, key);
            if ((grp & lt_mask) == 0)
                atomicAdd(&o.bins[count], (unsigned)__popc(grp));
        }
    }
}

template <bool BATCH, int OUT>
__device__ __forceinline__ void store_result(const EscapeArgs &a, const uint32_t *pal, uint32_t *hbins, int fr,
                                             uint32_t p, int count, int mi, unsigned lt_mask)
{
    const Frame &F = BATCH ? a.frames[fr] : a.single;
    if constexpr (OUT == 1) {
        reinterpret_cast<uint16_t *>(F.counts)[p] = (uint16_t)count;
        F.rgba[p] = pal[colour_index((uint32_t)count, (uint32_t)mi, F.colour_magic)];
        return;
    }
    if (F.counts) {
        if (F.count_type == JL_COUNT_U8)
            F.counts[p] = (uint8_t)count;
        else
            reinterpret_cast<uint16_t *>(F.counts)[p] = (uint16_t)count;
    }
    if (F.rgba)
        F.rgba[p] = pal[colour_index((uint32_t)count, (uint32_t)mi, F.colour_magic)];
    if (F.hist_bins) {
        if (!BATCH && a.hist_smem) {
            atomicAdd(&hbins[count], 1u);
        } else {
            const unsigned act = __activemask();
            const unsigned long long key = ((unsigned long long)(unsigned)fr << 32) | (unsigned)count;
            const unsigned grp = __match_any_sync(act, key);
            if ((grp & lt_mask) == 0)
                atomicAdd(&F.hist_bins[count], (unsigned)__popc(grp));
        }
    }
}

// ---------------------------------------------------------------------------
// Static kernel: one pixel per thread, CTA = 32 x 8 pixels (8 warps of 8 x 4),
// an exact test at every step and per-lane early exit.  No refill machinery,
// so per-pixel overhead is minimal; lanes of a warp wait for the slowest
// pixel of their 8 x 4 patch.  Best for frames with low escape counts.
// OUT (binary32 only): 1 = every frame has uint16 counts and RGBA8 and no
// histogram, 2 = every frame has RGBA8 only, 3 = every frame has uint8 counts
// and RGBA8 and no histogram; the stores then skip the per-frame output
// tests.  0: any outputs.
// ---------------------------------------------------------------------------
template <typename T, bool BATCH, int OUT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) escape_static_kernel(const __grid_constant__ EscapeArgs a)
{
    __shared__ uint32_t pal[256];
    extern __shared__ uint32_t hbins[];
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    // Tiles of 32 x 32 pixels in eight 8 x 16 parts; a warp takes parts one at
    // a time from the launch's counter (the next index fetched a part ahead).
    // In part k the warp covers 8 x 4 patches and each thread four pixels of
    // one column, 8 rows apart.
    const int lane = threadIdx.x & 31;
    const long long t_start = clock64();
    const long long total_units = a.total_tiles * 8;
    const unsigned long long claim = (unsigned long long)a.claim;
    unsigned long long next_u = 0;
    if (lane == 0)
        next_u = atomicAdd(a.chunk_counter, claim);
    long long cur = 0, end = 0;
    // next unit of this warp (warp-uniform; claims of `claim` units, the next
    // claim fetched one ahead)
    auto take_unit = [&]() -> long long {
        if (cur == end) {
            cur = (long long)__shfl_sync(FULL, next_u, 0);
            end = cur + (long long)claim;
            if (lane == 0)
                next_u = atomicAdd(a.chunk_counter, claim);
        }
        return cur++;
    };
    // batches: a unit's tile record (frame, index in the frame) is loaded one
    // unit ahead, so its latency overlaps the previous unit's work
    long long unit = take_unit();
    int f_cur = 0;
    uint32_t lt_cur = 0;
    if (BATCH && unit < total_units) {
        f_cur = a.tile_frame[unit >> 3];
        lt_cur = (uint32_t)a.tile_local[unit >> 3];
    }

    for (;;) {
        if (unit >= total_units)
            break;
        // budget check, uniform across the warp (the loop below has warp collectives)
        if (a.cycle_budget > 0 && __any_sync(FULL, (clock64() - t_start) > a.cycle_budget)) {
            if (lane == 0 && a.status)
                atomicExch(a.status, (int)JL_ETIMEOUT);
            break;
        }
        const long long nunit = take_unit();
        int f_nxt = 0;
        uint32_t lt_nxt = 0;
        if (BATCH && nunit < total_units) {
            f_nxt = a.tile_frame[nunit >> 3];
            lt_nxt = (uint32_t)a.tile_local[nunit >> 3];
        }
        const long long tile = unit >> 3;
        const int part = (int)(unit & 7);
        const int dx = (part & 3) * 8 + (lane & 7);
        const int dy = (part >> 2) * 4 + (lane >> 3);
        const int f = f_cur;
        const Frame &F = BATCH ? a.frames[f] : a.single;
        // frame fields used below, read once per tile
        const int W = F.W, H = F.H, mi = F.max_iter;
        const bool julia = F.mode == JL_JULIA;
        const bool safe = F.safe != 0;
        const T fcr = WorkT<T>::cr(F), fci = WorkT<T>::ci(F);
        const T *xs = static_cast<const T *>(F.xs);
        const T *ys = static_cast<const T *>(F.ys);
        TileOut o;
        o.counts = F.counts;
        o.rgba = F.rgba;
        o.bins = F.hist_bins;
        o.magic = F.colour_magic;
        o.m32 = (uint32_t)((o.magic - 1u) >> 8) + 1u;
        o.mi = mi;
        o.u8 = F.count_type == JL_COUNT_U8;
        o.small = mi <= 4096;
        const uint32_t lt = BATCH ? lt_cur : (uint32_t)(tile - F.tile_begin);
        const uint32_t ty = (uint32_t)(((uint64_t)lt * F.tiles_x_magic) >> 40);
        const uint32_t tx = lt - ty * (uint32_t)F.tiles_x;
        const int i = (int)tx * 32 + dx;
        if (i < W) {
            const T xv = xs[i];
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int j = (int)ty * 32 + dy + 8 * q;
                if (j >= H)
                    break;
                const T yv = ys[j];
                int count;
                if (julia)
                    count = escape_blocked(xv, yv, fcr, fci, mi, safe);
                else
                    count = escape_blocked(T(0), T(0), xv, yv, mi, !in_unsafe_band(xv, yv));
                store_tile<BATCH, OUT>(a, o, pal, hbins, f, (uint32_t)(j * W + i), count, (1u << lane) - 1u);
            }
        }
        unit = nunit;
        f_cur = f_nxt;
        lt_cur = lt_nxt;
    }
    if (nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const uint32_t v = hbins[t];
            if (v)
                atomicAdd(&a.single.hist_bins[t], v);
        }
    }
}

// S2: steps per block after the first 16 steps (super-blocks of 4 S2 steps).
// OUT = 1: every frame of the launch has uint16 counts and RGBA8 and no
// histogram (stores without per-frame tests); 0: any outputs.
template <bool BATCH, int S2, int OUT>
__global__ void __launch_bounds__(256, 4) escape_compact_kernel(const __grid_constant__ EscapeArgs a, int T)
{
    __shared__ uint32_t pal[256];
    __shared__ ParkRing rings[8];
    extern __shared__ uint32_t hbins[];
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    ParkRing &R = rings[w];
    const long long t_start = clock64();
    int qh = 0, qn = 0;  // ring head and fill (warp-uniform)
    bool stop = false;

    // Park the live lanes (state Z_n, C, n, pixel, frame) at the ring's tail.
    auto park = [&](unsigned m, bool &live, float x, float y, float cr, float ci, int n, int fr, uint32_t p) {
        if (live) {
            const int s = (qh + qn + __popc(m & lt_mask)) & (kQCap - 1);
            R.x[s] = x;
            R.y[s] = y;
            R.cr[s] = cr;
            R.ci[s] = ci;
            R.n[s] = n;
            R.f[s] = fr;
            R.p[s] = p;
            live = false;
        }
        qn += __popc(m);
        __syncwarp();
    };

    // Resume up to 32 parked pixels and run them until they finish or, when
    // few are left, park them again (`merge_only`: the tiles are done, park
    // only to merge with pixels already in the ring).
    auto resume = [&](bool merge_only) {
        float x = 0.f, y = 0.f, cr = 0.f, ci = 0.f;
        int n = 0, fr = 0, mi = 0, count = 0;
        uint32_t p = 0;
        bool live = false, fin = false;
        const int take = min(qn, 32);
        if (lane < take) {
            const int s = (qh + lane) & (kQCap - 1);
            x = R.x[s];
            y = R.y[s];
            cr = R.cr[s];
            ci = R.ci[s];
            n = R.n[s];
            fr = R.f[s];
            p = R.p[s];
            live = true;
            mi = (BATCH ? a.frames[fr] : a.single).max_iter;
        }
        qh = (qh + take) & (kQCap - 1);
        qn -= take;
        __syncwarp();
        for (int it = 0;; ++it) {
            if (live && n + 4 * S2 > mi) {
                count = escape_from(x, y, cr, ci, n, mi);
                live = false;
                fin = true;
            }
            const unsigned m = __ballot_sync(FULL, live);
            if (m == 0)
                break;
            const int nl = __popc(m);
            if (it > 0 && nl <= T && qn + nl <= kQCap && (!merge_only || qn > 0)) {
                park(m, live, x, y, cr, ci, n, fr, p);
                break;
            }
            if (live) {
                const int c = superblock<S2>(x, y, cr, ci, n);
                if (c < 0) {
                    n += 4 * S2;
                } else {
                    count = c;
                    live = false;
                    fin = true;
                }
            }
        }
        if (fin)
            store_result<BATCH, OUT>(a, pal, hbins, fr, p, count, mi, lt_mask);
    };

    // Work units: the eight 8 x 16 parts of every 32 x 32 tile (part k: columns
    // (k % 4) * 8 .. +7, rows (k / 4) * 4 + {0..3} + 8 q), taken one at a time
    // from the launch's counter; the next unit's index is fetched a unit ahead.
    const long long total_units = a.total_tiles * 8;
    const unsigned long long claim = (unsigned long long)a.claim;
    unsigned long long next_u = 0;
    if (lane == 0)
        next_u = atomicAdd(a.chunk_counter, claim);
    long long cur = 0, end = 0;
    for (;;) {
        if (cur == end) {
            cur = (long long)__shfl_sync(FULL, next_u, 0);
            end = cur + (long long)claim;
            if (lane == 0)
                next_u = atomicAdd(a.chunk_counter, claim);
        }
        const long long unit = cur++;
        if (unit >= total_units)
            break;
        if (a.cycle_budget > 0 && __any_sync(FULL, (clock64() - t_start) > a.cycle_budget)) {
            if (lane == 0 && a.status)
                atomicExch(a.status, (int)JL_ETIMEOUT);
            stop = true;
            break;
        }
        const long long tile = unit >> 3;
        const int part = (int)(unit & 7);
        const int dx = (part & 3) * 8 + (lane & 7);
        const int dy = (part >> 2) * 4 + (lane >> 3);
        int fr = 0;
        if constexpr (BATCH)
            fr = a.tile_frame[tile];
        const Frame &F = BATCH ? a.frames[fr] : a.single;
        const int W = F.W, H = F.H, mi = F.max_iter;
        const bool julia = F.mode == JL_JULIA;
        const bool safe = F.safe != 0;
        const float fcr = F.cr32, fci = F.ci32;
        const float *ys = static_cast<const float *>(F.ys);
        TileOut o;
        o.counts = F.counts;
        o.rgba = F.rgba;
        o.bins = F.hist_bins;
        o.magic = F.colour_magic;
        o.m32 = (uint32_t)((o.magic - 1u) >> 8) + 1u;
        o.mi = mi;
        o.u8 = F.count_type == JL_COUNT_U8;
        o.small = mi <= 4096;
        const uint32_t lt = BATCH ? (uint32_t)a.tile_local[tile] : (uint32_t)(tile - F.tile_begin);
        const uint32_t ty = (uint32_t)(((uint64_t)lt * F.tiles_x_magic) >> 40);
        const uint32_t tx = lt - ty * (uint32_t)F.tiles_x;
        const int i = (int)tx * 32 + dx;
        const float xv = i < W ? static_cast<const float *>(F.xs)[i] : 0.f;
        // Julia: Z_0 = pixel, C = frame constant; Mandelbrot: Z_0 = 0, C = pixel
        const float x0 = julia ? xv : 0.f;
        const float c0r = julia ? fcr : xv;
        // the straight-line first block needs 4 tests allowed and monotone escape
        // (Mandelbrot pixels in the unsafe band send their patch to the general path)
        const bool fast = mi >= 4 && (!julia || safe);
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            if (qn >= 32)
                resume(false);
            const int j = (int)ty * 32 + dy + 8 * q;
            const bool valid = i < W && j < H;
            if (!__any_sync(FULL, valid))
                break;  // rows beyond the frame: so are the later patches of this tile
            const float yv = ys[min(j, H - 1)];
            float x = x0, y = julia ? yv : 0.f;
            const float cr = c0r, ci = julia ? fci : yv;
            const uint32_t p = (uint32_t)j * (uint32_t)W + (uint32_t)i;
            bool live = valid, fin = false;
            int count = 0;
            int n0 = 0;  // steps already run by every live lane
            if (fast) {
                // Straight-line first block: 4 steps for every lane, one vote.
                // In about two thirds of the patches of typical frames every
                // pixel has failed a test by then (the far field) and the
                // patch is done here; otherwise the live pixels go on from
                // Z_4 on the general path below.
                const float r0 = step32(x, y, cr, ci);
                const float r1 = step32(x, y, cr, ci);
                const float r2 = step32(x, y, cr, ci);
                const float r3 = step32(x, y, cr, ci);
                const bool hold = r3 <= 4.0f;
                const bool unsafe = !julia && in_unsafe_band(cr, ci);
                if (__ballot_sync(FULL, valid && (hold || unsafe)) == 0) {
                    if (valid)
                        store_tile<BATCH, OUT>(a, o, pal, hbins, fr, p, (r0 <= 4.0f) + (r1 <= 4.0f) + (r2 <= 4.0f),
                                               lt_mask);
                    continue;
                }
                if (valid && unsafe) {
                    // escape not proven monotone: exact single steps from Z_0
                    count = exact_from(x0, julia ? yv : 0.f, cr, ci, 0, mi);
                    live = false;
                    fin = true;
                } else if (valid && !hold) {
                    count = (r0 <= 4.0f) + (r1 <= 4.0f) + (r2 <= 4.0f);
                    live = false;
                    fin = true;
                }
                n0 = 4;
            } else if (!julia) {
                // pixels whose escape is not proven monotone: exact single steps
                const bool unsafe = valid && in_unsafe_band(cr, ci);
                if (__any_sync(FULL, unsafe) && unsafe) {
                    count = exact_from(x, y, cr, ci, 0, mi);
                    live = false;
                    fin = true;
                }
            } else if (!safe && valid) {
                count = exact_from(x, y, cr, ci, 0, mi);
                live = false;
                fin = true;
            }
            if (mi < n0 + 16) {
                if (live) {
                    count = escape_from(x, y, cr, ci, n0, mi);
                    live = false;
                    fin = true;
                }
            } else {
                // 16 steps in blocks of 4 (most of the remaining pixels leave
                // here), then super-blocks of 32 steps in blocks of 8; n is the
                // same for every live lane of the patch
                if (live) {
                    const int c = superblock<4>(x, y, cr, ci, n0);
                    if (c >= 0) {
                        count = c;
                        live = false;
                        fin = true;
                    }
                }
                int n = n0 + 16;
                for (;;) {
                    const unsigned m = __ballot_sync(FULL, live);
                    if (m == 0)
                        break;
                    const int nl = __popc(m);
                    if (nl <= T && qn + nl <= kQCap) {
                        park(m, live, x, y, cr, ci, n, fr, p);
                        break;
                    }
                    if (n + 4 * S2 > mi) {
                        if (live) {
                            count = escape_from(x, y, cr, ci, n, mi);
                            live = false;
                            fin = true;
                        }
                        break;
                    }
                    if (live) {
                        const int c = superblock<S2>(x, y, cr, ci, n);
                        if (c >= 0) {
                            count = c;
                            live = false;
                            fin = true;
                        }
                    }
                    n += 4 * S2;
                }
            }
            if (fin)
                store_tile<BATCH, OUT>(a, o, pal, hbins, fr, p, count, lt_mask);
        }
    }
    // the tiles are done: finish the parked pixels, merging partial batches
    while (qn > 0 && !stop)
        resume(true);

    if (nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const uint32_t v = hbins[t];
            if (v)
                atomicAdd(&a.single.hist_bins[t], v);
        }
    }
}

// ---------------------------------------------------------------------------
// Certified binary32 pass for binary64 frames.
//
// A binary64 frame's counts are those of the binary64 orbit Z_{n+1} = Z_n^2 + C
// (round to nearest, no FMA) with the test x2 + y2 > 4 taken in binary64, and
// the binary64 pipe of this part issues ~74x fewer operations per clock than
// the binary32 one.  This pass runs a binary32 orbit W_n beside that orbit with
// a running bound E_n >= |Z_n - W_n| (complex modulus) and takes a binary64 test
// from binary32 values only where the bound settles it:
//     (|W| - E)^2 <= |Z|^2 <= (|W| + E)^2.
// A certified test is the binary64 test's own outcome, so a pixel whose tests
// are all certified, up to its escape or to the limit, gets exactly its
// binary64 count.  A pixel with a test the bound cannot settle goes to a list
// that the binary64 kernel (LIST) renders from Z_0.
//
// u = 2^-24.  The orbit is rounded to nearest; the bound arithmetic rounds
// toward +inf (toward -inf for the lower bound), so it never understates.
//   orbit   y2 = y*y, r = fma(x, x, y2), x' = fma(x, x, fma(-y, y, cr)),
//           y' = fma(x + x, y, ci);  |W|^2 is within r (1 +- 2^-20)
//   modulus s = sqrt.approx(r) (1 + 2^-10) >= |W|  (the PTX approximation is
//           within ~2^-23 relative; the factor leaves 2^10 of room)
//   pass    U = r (1 + 2^-20) + E (2 s + E) + EC < 4  =>  binary64 x2 + y2 <= 4
//           (U <= 4 - 2^-22, and the binary64 sum of squares is within 2^-51
//           of |Z|^2 relative)
//   escape  L = r (1 - 2^-20) - 2 s E > 4  =>  binary64 x2 + y2 > 4
//   bound   E' = E (2 s + E) + EC + 2.5 u r
// The new bound adds up |Z^2 - W^2| <= E (2|W| + E); |C - C32|_1; the binary32
// rounding of the step, at most u (1 + 2^-19)(|x'| + |y'| + |cr| + y2) in the
// 1-norm, which is <= 2.5 u r + u (1 + 2^-19)(2|cr| + |ci|) because
// |x'| + |y'| <= sqrt(2) |W|^2 + |C|_1 to first order; and the binary64
// rounding of the step, <= 2^-48 + 2^-52 |C|_1 while |Z|^2 <= 4, plus underflow
// terms below 2^-146.  EC collects the terms that do not depend on W:
//   Julia:      EC = |C - C32|_1 + 2^-22 (|cr32| + |ci32|) + 2^-47 for the frame
//               (`cert_error_constant`); E_0 = u (1 + 2^-20)(|x| + |y|) + 2^-140,
//               the rounding of the pixel's coordinates;
//   Mandelbrot: C32 is the pixel, E_0 = 0 (Z_0 = 0 on both sides) and
//               EC = 3 u (1 + 2^-18)(|cr| + |ci|) + 2^-47.
// A NaN or infinity anywhere makes both tests false: the pixel goes to the list.
// ---------------------------------------------------------------------------
static constexpr float kCertS2 = 0x1.004p+1f;     // 2 (1 + 2^-10)
static constexpr float kCertR1 = 0x1.00001p+0f;   // 1 + 2^-20
static constexpr float kCertR0 = 0x1.ffffep-1f;   // 1 - 2^-20
static constexpr float kCertK2 = 0x1.4p-23f;      // 2.5 u
static constexpr float kCertE0 = 0x1.00001p-24f;  // u (1 + 2^-20)
static constexpr float kCertMC = 0x1.80006p-23f;  // 3 u (1 + 2^-18)

float cert_error_constant(double cr, double ci, float cr32, float ci32)
{
    const double v = (fabs(cr - (double)cr32) + fabs(ci - (double)ci32) +
                      0x1p-22 * (fabs((double)cr32) + fabs((double)ci32)) + 0x1p-47) * (1.0 + 0x1p-40);
    float f = (float)v;
    if ((double)f < v)
        f = nextafterf(f, INFINITY);
    return f;
}

// Approximate square root with subnormal inputs flushed to zero (the form
// without flushing spends extra instructions on subnormals: the binary32 pass
// 3.27 -> 2.76 ms with this one).  A flushed r < 2^-126 gives s = 0 although
// |W| may be up to 2^-62: the omitted 2 |W| E is below 2^-60 E, within the
// slack of the passes' constants (EC >= 2^-47 of which the binary64 step's
// rounding takes 2^-48; the double-float test's 2^-58), and a test with E or
// Et above 2 does not pass anyway; the escape test L needs r > 4 and is not
// affected.
__device__ __forceinline__ float sqrt_approx(float r)
{
    float s;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(r));
    return s;
}

// One certified step from (W_n, E_n): 1 = the binary64 test of Z_n passed
// (the state then holds W_{n+1}, E_{n+1}); 0 = it failed (escape at n);
// -1 = not settled by the bound.
__device__ __forceinline__ int cert_step(float &x, float &y, float &e, float cr, float ci, float ec)
{
    const float y2 = __fmul_rn(y, y);
    const float r = __fmaf_rn(x, x, y2);
    const float s = sqrt_approx(r);
    const float ge = __fmaf_ru(e, __fmaf_ru(kCertS2, s, e), ec);
    if (__fmaf_ru(r, kCertR1, ge) < 4.0f) {
        const float nx = __fmaf_rn(x, x, __fmaf_rn(-y, y, cr));
        y = __fmaf_rn(__fadd_rn(x, x), y, ci);
        x = nx;
        e = __fmaf_ru(kCertK2, r, ge);
        return 1;
    }
    const float m = __fmul_ru(__fmul_ru(kCertS2, s), e);
    return __fmaf_rd(r, kCertR0, -m) > 4.0f ? 0 : -1;
}

// Escape certified from a step's kept values (r, s, E): 0 = escape, -1 = not settled.
__device__ __forceinline__ int cert_exit(float r, float s, float e)
{
    const float m = __fmul_ru(__fmul_ru(kCertS2, s), e);
    return __fmaf_rd(r, kCertR0, -m) > 4.0f ? 0 : -1;
}

// One block of CB certified steps; false (state restored to the block's
// start) when its test is not a certified pass.  The largest U of the block is
// compared with 4 (a NaN U cannot come first: with finite inputs r, s and g
// are finite or +inf and E > 0 after step 0 (E_0 = 0 only with W_0 = 0), so the
// first U that is not finite is +inf, which the maximum keeps).
//
// MONO: only the block's last U is formed.  With B_n = |W_n| + E_n, the
// update of E adds at least E (2|W| + E) and the bound on the binary32 step's
// rounding, so B_{n+1} >= B_n^2 - |C32| for the computed values, whatever Z
// does.  If the first binary64 test to fail is test m, E_m still bounds
// |Z_m - W_m| (the tests before m passed), so B_m >= |Z_m| > 2 - 2^-50:
// with |C32| <= 2 - 2^-12, B_{m+1} > 2 + 2^-13 and B stays above 2, so every
// later U >= B^2 > 4, and U_m >= 4 by the test's own certificate.  Hence a
// last U < 4 certifies every test of the block.  For Mandelbrot pixels with
// |C32| >= 2 (W_0 = 0, W_1 = C32), B_n >= |C32| for all n >= 1, so the first
// block's last U > 4 and its replay finds the escape at test 1.  The omitted
// 2 |W| E of a flushed subnormal r (below 2^-61 B) leaves B_{n+1} > 2 here.
// A NaN or infinite last U fails the compare and replays the block.
template <int CB, bool MONO>
__device__ __forceinline__ bool cert_block(float &x, float &y, float &e, float cr, float ci, float ec)
{
    const float x0 = x, y0 = y, e0 = e;
    float umax = 0.f;
#pragma unroll
    for (int u = 0; u < CB; ++u) {
        const float y2 = __fmul_rn(y, y);
        const float r = __fmaf_rn(x, x, y2);
        const float s = sqrt_approx(r);
        const float ge = __fmaf_ru(e, __fmaf_ru(kCertS2, s, e), ec);
        if (!MONO)
            umax = fmaxf(umax, __fmaf_ru(r, kCertR1, ge));
        else if (u == CB - 1)
            umax = __fmaf_ru(r, kCertR1, ge);
        const float nx = __fmaf_rn(x, x, __fmaf_rn(-y, y, cr));
        y = __fmaf_rn(__fadd_rn(x, x), y, ci);
        x = nx;
        e = __fmaf_ru(kCertK2, r, ge);
    }
    if (umax < 4.0f)
        return true;
    x = x0;
    y = y0;
    e = e0;
    return false;
}

// Binary64 count of a pixel from the certified pass (tests n = 0 .. mi-1 from
// W_0 = (x, y), E_0 = e), or -1 - n when test n is not settled.  A first block
// of CB0 steps (shorter blocks waste fewer steps on the many pixels that
// escape within the first few tests), then blocks of CB (sweep pass 2.54 ms
// with blocks of 6 throughout, 2.52 with a first block of 2, 2.51 with 3); the
// block whose test is not a certified pass, and the tests after the last full
// block, run one test at a time.
template <int CB0, int CB, bool MONO>
__device__ __forceinline__ int cert_count(float x, float y, float e, float cr, float ci, float ec, int mi)
{
    int n = 0;
    bool ok = true;
    if (CB0 != CB && CB0 <= mi) {
        ok = cert_block<CB0, MONO>(x, y, e, cr, ci, ec);
        if (ok)
            n = CB0;
    }
    if (ok)
        for (; n + CB <= mi; n += CB)
            if (!cert_block<CB, MONO>(x, y, e, cr, ci, ec))
                break;
    for (; n < mi; ++n) {
        const int rc = cert_step(x, y, e, cr, ci, ec);
        if (rc <= 0)
            return rc == 0 ? n : -1 - n;
    }
    return mi;
}

// Tile kernel of the certified pass: the static kernel's 32 x 32 tiles, 8 x 16
// parts claimed from the launch counter, 8 x 4 patches.  Certified pixels are
// stored; the others are appended to the list, one counter increment per
// patch.  A list that is full (never, when cert_cap >= the launch's pixels)
// leaves its pixel to exact binary64 steps here.
template <bool BATCH, int OUT>
__global__ void __launch_bounds__(256, 4) cert_kernel(const __grid_constant__ EscapeArgs a)
{
    __shared__ uint32_t pal[256];
    extern __shared__ uint32_t hbins[];
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned steps = 0;  // tests this thread decided
    const long long t_start = clock64();
    const long long total_units = a.total_tiles * 8;
    const unsigned long long claim = (unsigned long long)a.claim;
    unsigned long long next_u = 0;
    if (lane == 0)
        next_u = atomicAdd(a.chunk_counter, claim);
    long long cur = 0, end = 0;
    for (;;) {
        if (cur == end) {
            cur = (long long)__shfl_sync(FULL, next_u, 0);
            end = cur + (long long)claim;
            if (lane == 0)
                next_u = atomicAdd(a.chunk_counter, claim);
        }
        const long long unit = cur++;
        if (unit >= total_units)
            break;
        if (a.cycle_budget > 0 && __any_sync(FULL, (clock64() - t_start) > a.cycle_budget)) {
            if (lane == 0 && a.status)
                atomicExch(a.status, (int)JL_ETIMEOUT);
            break;
        }
        const long long tile = unit >> 3;
        const int part = (int)(unit & 7);
        const int dx = (part & 3) * 8 + (lane & 7);
        const int dy = (part >> 2) * 4 + (lane >> 3);
        int fr = 0;
        if constexpr (BATCH)
            fr = a.tile_frame[tile];
        const Frame &F = BATCH ? a.frames[fr] : a.single;
        const int W = F.W, H = F.H, mi = F.max_iter;
        const bool julia = F.mode == JL_JULIA;
        const float fcr = F.cr32, fci = F.ci32, fec = F.cert_ec;
        const float *xs32 = F.xs32;
        const float *ys32 = F.ys32;
        TileOut o;
        o.counts = F.counts;
        o.rgba = F.rgba;
        o.bins = F.hist_bins;
        o.magic = F.colour_magic;
        o.m32 = (uint32_t)((o.magic - 1u) >> 8) + 1u;
        o.mi = mi;
        o.u8 = F.count_type == JL_COUNT_U8;
        o.small = mi <= 4096;
        const uint32_t lt = BATCH ? (uint32_t)a.tile_local[tile] : (uint32_t)(tile - F.tile_begin);
        const uint32_t ty = (uint32_t)(((uint64_t)lt * F.tiles_x_magic) >> 40);
        const uint32_t tx = lt - ty * (uint32_t)F.tiles_x;
        const int i = (int)tx * 32 + dx;
        const float xv = i < W ? xs32[i] : 0.f;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int j = (int)ty * 32 + dy + 8 * q;
            const bool valid = i < W && j < H;
            if (!__any_sync(FULL, valid))
                break;  // rows beyond the frame: so are the later patches of this tile
            int count = 0;
            if (valid) {
                const float yv = ys32[j];
                const float ax = fabsf(xv), ay = fabsf(yv);
                if (julia) {
                    const float e0 = __fmaf_ru(kCertE0, __fadd_ru(ax, ay), 0x1p-140f);
                    count = F.safe ? cert_count<3, 6, true>(xv, yv, e0, fcr, fci, fec, mi)
                                   : cert_count<4, 4, false>(xv, yv, e0, fcr, fci, fec, mi);
                } else {
                    // (a pixel outside the band |C|^2 in (3.99, 4.01) has |C32| <= 2 - 2^-12 or >= 2)
                    const float ec = __fmaf_ru(kCertMC, __fadd_ru(ax, ay), 0x1p-47f);
                    count = !in_unsafe_band(xv, yv) ? cert_count<3, 6, true>(0.f, 0.f, 0.f, xv, yv, ec, mi)
                                                    : cert_count<4, 4, false>(0.f, 0.f, 0.f, xv, yv, ec, mi);
                }
            }
            const bool undecided = valid && count < 0;
            // tests decided (for the launch's step counter)
            if (valid)
                steps += count < 0 ? (unsigned)(-count) : (unsigned)(count < mi ? count + 1 : mi);
            const unsigned um = __ballot_sync(FULL, undecided);
            unsigned long long base = 0;
            if (um) {
                if (lane == 0)
                    base = atomicAdd(a.cert_count, (unsigned long long)__popc(um));
                base = __shfl_sync(FULL, base, 0);
            }
            if (undecided) {
                const unsigned long long k = base + (unsigned long long)__popc(um & lt_mask);
                if (k < (unsigned long long)a.cert_cap) {
                    a.cert_list[k] = ((uint64_t)(uint32_t)fr << 32) | ((uint64_t)(uint32_t)j << 16) | (uint32_t)i;
                    continue;
                }
                // no room in the list: exact binary64 steps here
                const double x64 = static_cast<const double *>(F.xs)[i];
                const double y64 = static_cast<const double *>(F.ys)[j];
                count = julia ? exact_from(x64, y64, F.cr, F.ci, 0, mi) : exact_from(0.0, 0.0, x64, y64, 0, mi);
            }
            if (valid)
                store_tile<BATCH, OUT>(a, o, pal, hbins, fr, (uint32_t)j * (uint32_t)W + (uint32_t)i, count, lt_mask);
        }
    }
    if (a.cert_steps) {
        const unsigned tot = __reduce_add_sync(FULL, steps);
        if (lane == 0)
            atomicAdd(a.cert_steps, (unsigned long long)tot);
    }
    if (nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const uint32_t v = hbins[t];
            if (v)
                atomicAdd(&a.single.hist_bins[t], v);
        }
    }
}

// ---------------------------------------------------------------------------
// Second certified pass: double-float orbit over the binary32 pass's list.
//
// The pixels the binary32 pass cannot settle are mostly escaping pixels whose
// orbits stay long near the Julia set: the distance bound grows with the
// derivative of the iterate and reaches the test's margin after ~200 steps.
// This pass carries W as pairs of binary32 values (x = xh + xl, ~48 bits) so
// that the bound starts and grows ~2^24 times lower, with the same rule: a
// test is decided from W only when [(|W| - E)^2, (|W| + E)^2] lies on one side
// of 4, and a pixel with an unsettled test goes on to the binary64 kernel.
//
// Step (u = 2^-24; every operation round to nearest, products split exactly
// with FMA: a*b = p + e, e = fma(a, b, -p); sums of two values split exactly
// by TwoSum (6 operations) where the exact rounding error is needed):
//   x^2 - y^2 + cr:  TwoSum(p1 - p2) -> (t, et), TwoSum(t + crh) -> (sx, esx),
//                    lx = ((fma(-2yh, yl, fma(2xh, xl, crl)) + (e1 - e2)) + et) + esx
//   2xy + ci:        TwoSum(2 p3 + cih) -> (sy, esy),
//                    ly = fma(2, e3, fma(2xl, yh, fma(2xh, yl, cil))) + esy
//   renormalised:    (xh', xl') = TwoSum(sx + lx), (yh', yl') = TwoSum(sy + ly)
// Exact real and imaginary parts differ from sx + lx and sy + ly only by the
// roundings of the ten low-part operations (each at most u times the
// magnitude of its terms) and the dropped xl^2 - yl^2 and 2 xl yl.  With
// Lambda = |xl| + |yl| and |xh| + |yh| <= 2 sqrt(2) (|Wh| < 2 after a pass):
//   delta <= 6.01 u (2 (|xh| + |yh|) Lambda + |Cl|_1 + u (20.1 + |Ch|_1)) + Lambda^2
//         <= Lambda (36 u + Lambda) + 6.01 u |Cl|_1 + 6.01 u^2 (20.1 + |Ch|_1) + 2^-145
// (the e terms are at most u times their products and sums, |t|, p1 + p2 and
// 2|p3| <= |Wh|^2 < 4, |sx| + |sy| <= 8 + |Ch|_1).  Test: Wh = xh + i yh is
// within Et = E + Lambda of Z, and the binary32 pass's test applies to
// (Wh, Et).  Bound: E' = E (2 (s + Lambda) + E) + delta + |C - Cdf|_1 +
// binary64 step rounding (2^-48 + 2^-52 |C|_1).  KC collects the W-independent
// terms: per frame for Julia (`cert2_frame_constants`), per pixel for
// Mandelbrot (C = the pixel as a float pair).  Initial E: the pixel's
// coordinates as float pairs, u (1 + 2^-20) Lambda_0 + 2^-140 (Julia), 0
// (Mandelbrot: Z_0 = 0).
// ---------------------------------------------------------------------------
static constexpr int kDfBlock = 16;           // steps per block of the double-float pass
static constexpr float kDfKL = 0x1.2p-19f;    // 36 u
static constexpr float kDfMl = 0x1.dp-22f;    // 7.25 u: Mandelbrot KC per unit of |Cl|_1
static constexpr float kDfMh = 0x1.9p-46f;    // 6.25 u^2: Mandelbrot KC per unit of |Ch|_1
static constexpr float kDfM0 = 0x1p-41f;      // 128 u^2: Mandelbrot KC constant

void cert2_frame_constants(double cr, double ci, float cr32, float ci32, float *cr_lo, float *ci_lo, float *kc)
{
    // cr - cr32 is exact (Sterbenz); so is its difference with its own rounding
    const double dr = cr - (double)cr32, di = ci - (double)ci32;
    *cr_lo = (float)dr;
    *ci_lo = (float)di;
    const double u = 0x1p-24;
    const double dC = fabs(dr - (double)*cr_lo) + fabs(di - (double)*ci_lo);
    const double ah = fabs((double)cr32) + fabs((double)ci32), al = fabs((double)*cr_lo) + fabs((double)*ci_lo);
    const double v = (6.01 * u * al + 6.01 * u * u * (20.1 + ah) + dC + 0x1p-48 + 0x1.03p-52 * (ah + al) +
                      0x1p-139) * (1.0 + 0x1p-40);
    float f = (float)v;
    if ((double)f < v)
        f = nextafterf(f, INFINITY);
    *kc = f;
}

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// State of the double-float pass for one pixel.
struct DfState {
    float xh, xl, yh, yl, e;
};

// One double-float step with its bound update (after a certified pass); the
// new pairs are renormalised by TwoSum.
__device__ __forceinline__ void df_update(DfState &w, float s, float lam, float crh, float crl, float cih, float cil,
                                          float kc)
{
    const float p1 = __fmul_rn(w.xh, w.xh), e1 = __fmaf_rn(w.xh, w.xh, -p1);
    const float p2 = __fmul_rn(w.yh, w.yh), e2 = __fmaf_rn(w.yh, w.yh, -p2);
    const float p3 = __fmul_rn(w.xh, w.yh), e3 = __fmaf_rn(w.xh, w.yh, -p3);
    float t, et, sx, esx, sy, esy;
    two_sum(p1, -p2, t, et);
    two_sum(t, crh, sx, esx);
    two_sum(__fadd_rn(p3, p3), cih, sy, esy);
    const float x2 = __fadd_rn(w.xh, w.xh), y2 = __fadd_rn(w.yh, w.yh);
    float lx = __fmaf_rn(-y2, w.yl, __fmaf_rn(x2, w.xl, crl));
    lx = __fadd_rn(__fadd_rn(__fadd_rn(lx, __fsub_rn(e1, e2)), et), esx);
    float ly = __fmaf_rn(2.0f, e3, __fmaf_rn(__fadd_rn(w.xl, w.xl), w.yh, __fmaf_rn(x2, w.yl, cil)));
    ly = __fadd_rn(ly, esy);
    // bound first (it uses the old E and Lambda)
    const float g2 = __fmaf_ru(kCertS2, s, __fmaf_ru(2.0f, lam, w.e));
    w.e = __fmaf_ru(w.e, g2, __fmaf_ru(lam, __fadd_ru(kDfKL, lam), kc));
    two_sum(sx, lx, w.xh, w.xl);
    two_sum(sy, ly, w.yh, w.yl);
}

// Up to NB tests of the double-float pass from test n (limit mi): the
// pixel's count (>= 0) when settled, -1 when a test is not settled, -2 when
// the tests passed so far leave it live (n advanced).  NB steps always run
// (the state after a failed or an uncounted test is not used again); each
// keeps its test's r, s and Et, so the first test that is not a certified
// pass is classified from those without running the block again.  The
// pixels of this pass live for ~200 steps, so long blocks pay: per block a
// round of refills, stores and list appends with few lanes active (sweep
// pass 3.01 ms with blocks of 4, 2.64 with 8, 2.42 with 16, 2.39 with 24,
// 2.72 with 32).
template <int NB>
__device__ __forceinline__ int df_run(DfState &w, int &n, int mi, float crh, float crl, float cih, float cil, float kc)
{
    if (n >= mi)
        return mi;
    float rk[NB], sk[NB], ek[NB];
    bool pk[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const float lam = __fadd_ru(fabsf(w.xl), fabsf(w.yl));
        const float et = __fadd_ru(w.e, lam);
        const float r = __fmaf_rn(w.xh, w.xh, __fmul_rn(w.yh, w.yh));
        const float s = sqrt_approx(r);
        const float ge = __fmaf_ru(et, __fmaf_ru(kCertS2, s, et), 0x1p-58f);
        pk[k] = __fmaf_ru(r, kCertR1, ge) < 4.0f;
        rk[k] = r;
        sk[k] = s;
        ek[k] = et;
        df_update(w, s, lam, crh, crl, cih, cil, kc);
    }
    const int m = min(NB, mi - n);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (k < m && !pk[k]) {
            if (cert_exit(rk[k], sk[k], ek[k]) == 0)
                return n + k;
            n += k;  // the test that is not settled
            return -1;
        }
    }
    n += m;
    return n >= mi ? mi : -2;
}

// Lane-refill kernel of the double-float pass: warps take 32-entry pieces of
// the binary32 pass's list from *list2_counter; a lane whose pixel is settled
// (stored) or not settled (appended to cert_list2, one counter increment per
// warp and round of blocks) takes the next entry of its warp's piece.  A full
// second list (never, when cert_cap >= the launch's pixels) leaves its pixel
// to exact binary64 steps here.
template <bool BATCH, int OUT>
__global__ void __launch_bounds__(256) cert2_kernel(const __grid_constant__ EscapeArgs a)
{
    __shared__ uint32_t pal[256];
    extern __shared__ uint32_t hbins[];
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = (!BATCH && a.hist_smem) ? a.single.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned steps = 0;  // tests this thread decided
    const long long t_start = clock64();
    long long n1 = (long long)*a.cert_count;
    if (n1 > a.cert_cap)
        n1 = a.cert_cap;
    const long long pieces = (n1 + 31) >> 5;
    unsigned long long next_c = 0;
    if (lane == 0)
        next_c = atomicAdd(a.list2_counter, 1ull);
    long long q_base = 0;
    int q_pos = 0, q_end = 0;
    bool q_done = false;

    DfState w{0.f, 0.f, 0.f, 0.f, 0.f};
    float crh = 0.f, crl = 0.f, cih = 0.f, cil = 0.f, kc = 0.f;
    int n = 0, mi = 0, fr = 0, pi = 0, pj = 0;
    bool live = false;

    for (;;) {
        // refill the lanes without a pixel from the warp's piece of the list
        unsigned want = __ballot_sync(FULL, !live);
        while (want && !q_done) {
            if (q_pos >= q_end) {
                const unsigned long long c = __shfl_sync(FULL, next_c, 0);
                bool over = a.cycle_budget > 0 && (clock64() - t_start) > a.cycle_budget;
                over = __any_sync(FULL, over);
                if ((long long)c >= pieces || over) {
                    if (over && lane == 0 && a.status && (long long)c < pieces)
                        atomicExch(a.status, (int)JL_ETIMEOUT);
                    q_done = true;
                    break;
                }
                if (lane == 0)
                    next_c = atomicAdd(a.list2_counter, 1ull);
                q_base = (long long)c << 5;
                q_pos = 0;
                q_end = (int)min(32ll, n1 - q_base);
                continue;
            }
            const int take = min(q_end - q_pos, __popc(want));
            const int rank = __popc(want & lt_mask);
            const bool got = ((want >> lane) & 1u) && rank < take;
            if (got) {
                const uint64_t ent = a.cert_list[q_base + q_pos + rank];
                fr = (int)(ent >> 32);
                pj = (int)((ent >> 16) & 0xffffu);
                pi = (int)(ent & 0xffffu);
                const Frame &F = BATCH ? a.frames[fr] : a.single;
                // the coordinates as float pairs (tables written with the binary64 ones)
                const float xh = F.xs32[pi], yh = F.ys32[pj];
                const float xl = F.xs32lo[pi], yl = F.ys32lo[pj];
                const float l0 = __fadd_ru(fabsf(xl), fabsf(yl));
                mi = F.max_iter;
                n = 0;
                if (F.mode == JL_JULIA) {
                    w = DfState{xh, xl, yh, yl, __fmaf_ru(kCertE0, l0, 0x1p-140f)};
                    crh = F.cr32;
                    crl = F.cr_lo32;
                    cih = F.ci32;
                    cil = F.ci_lo32;
                    kc = F.cert2_kc;
                } else {
                    w = DfState{0.f, 0.f, 0.f, 0.f, 0.f};
                    crh = xh;
                    crl = xl;
                    cih = yh;
                    cil = yl;
                    kc = __fmaf_ru(kDfMl, l0, __fmaf_ru(kDfMh, __fadd_ru(fabsf(xh), fabsf(yh)), kDfM0));
                }
                live = true;
            }
            want &= ~__ballot_sync(FULL, got);
            q_pos += take;
        }
        if (!__any_sync(FULL, live))
            break;
        int res = -2;
        if (live)
            res = df_run<kDfBlock>(w, n, mi, crh, crl, cih, cil, kc);
        const bool und = live && res == -1;
        if (live && res != -2)
            steps += res >= 0 ? (unsigned)(res < mi ? res + 1 : mi) : (unsigned)(n + 1);
        const unsigned um = __ballot_sync(FULL, und);
        if (um) {
            unsigned long long base = 0;
            if (lane == 0)
                base = atomicAdd(a.cert_count2, (unsigned long long)__popc(um));
            base = __shfl_sync(FULL, base, 0);
            if (und) {
                const unsigned long long k = base + (unsigned long long)__popc(um & lt_mask);
                if (k < (unsigned long long)a.cert_cap) {
                    a.cert_list2[k] = ((uint64_t)(uint32_t)fr << 32) | ((uint64_t)(uint32_t)pj << 16) | (uint32_t)pi;
                } else {
                    // no room in the second list: exact binary64 steps here
                    const Frame &F = BATCH ? a.frames[fr] : a.single;
                    const double x64 = static_cast<const double *>(F.xs)[pi];
                    const double y64 = static_cast<const double *>(F.ys)[pj];
                    res = F.mode == JL_JULIA ? exact_from(x64, y64, F.cr, F.ci, 0, mi)
                                             : exact_from(0.0, 0.0, x64, y64, 0, mi);
                }
            }
        }
        if (live && res >= 0) {
            const Frame &F = BATCH ? a.frames[fr] : a.single;
            store_result<BATCH, OUT>(a, pal, hbins, fr, (uint32_t)pj * (uint32_t)F.W + (uint32_t)pi, res, mi, lt_mask);
            if (a.cert2_iters) {
                const unsigned act = __activemask();
                const unsigned tot = __reduce_add_sync(act, (unsigned)res);
                if ((act & lt_mask) == 0)
                    atomicAdd(a.cert2_iters, (unsigned long long)tot);
            }
        }
        if (res != -2)
            live = false;
    }
    if (a.cert2_steps) {
        const unsigned tot = __reduce_add_sync(FULL, steps);
        if (lane == 0)
            atomicAdd(a.cert2_steps, (unsigned long long)tot);
    }
    if (nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const uint32_t v = hbins[t];
            if (v)
                atomicAdd(&a.single.hist_bins[t], v);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Resident CTAs per SM of a kernel for a block size and dynamic shared
// memory, asked of the runtime once per (device, kernel, threads, bytes): the
// query costs microseconds of host time, which would otherwise be paid on
// every small render.
cudaError_t occupancy_per_sm(const void *kern, int threads, size_t smem, int *out)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const auto key = std::make_tuple(dev, kern, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = per_sm;
    *out = per_sm;
    return cudaSuccess;
}

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_coords(const Frame *frames_dev, const Frame *single, int n, cudaStream_t st)
{
    CoordArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = frames_dev;
    a.n_frames = n;
    if (single)
        a.single = *single;
    coords_kernel<<<2 * n, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hist_finalize(const Frame *frames_dev, const Frame *single, int n, cudaStream_t st)
{
    HistArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = frames_dev;
    a.n_frames = n;
    if (single)
        a.single = *single;
    int grid = n < 4096 ? n : 4096;
    hist_finalize_kernel<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hist_zero(const Frame *frames_dev, int n, cudaStream_t st)
{
    HistArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = frames_dev;
    a.n_frames = n;
    int grid = n < 4096 ? n : 4096;
    hist_zero_kernel<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int PPT, int U, bool LIST = false>
static cudaError_t launch_one(const EscapeArgs &a, const Variant &v, int num_sms, size_t smem, cudaStream_t st)
{
    auto kern = a.frames ? escape_kernel<T, PPT, U, true, LIST> : escape_kernel<T, PPT, U, false, LIST>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    int per_sm = v.ctas_per_sm;
    if (per_sm <= 0) {
        cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), v.threads, smem, &per_sm);
        if (e != cudaSuccess)
            return e;
        if (per_sm < 1)
            per_sm = 1;
    }
    long long grid = (long long)num_sms * per_sm;
    // never more warps than chunks (the list's length is known only on the device)
    long long max_ctas = (a.total_chunks + (v.threads / 32) - 1) / (v.threads / 32);
    if (!LIST && grid > max_ctas)
        grid = max_ctas;
    if (grid < 1)
        grid = 1;
    kern<<<(unsigned)grid, v.threads, smem, st>>>(a);
    return cudaGetLastError();
}

#define JL_VARIANTS_F32(X) X(float, 1, 8) X(float, 2, 8) X(float, 4, 8) X(float, 2, 16) X(float, 4, 4) X(float, 8, 4)
// (binary64: the default shape first; the tuner keeps an earlier candidate
// unless a later one is more than 1 % faster)
#define JL_VARIANTS_F64(X) X(double, 4, 8) X(double, 2, 4) X(double, 1, 4) X(double, 2, 8) X(double, 4, 4) X(double, 1, 8)

bool variant_supported(int precision, int ppt, int unroll)
{
    if (ppt == 0 && unroll == 0 && (precision == JL_FP32 || precision == JL_FP64))
        return true;
    // (0, T): the compacting tile kernel (binary32), parking threshold T lanes
    if (ppt == 0 && precision == JL_FP32 && unroll >= 1 && unroll <= 32)
        return true;
#define JL_CHECK(T, P, UU) \
    if (((sizeof(T) == 8) == (precision == JL_FP64)) && ppt == P && unroll == UU) return true;
    JL_VARIANTS_F32(JL_CHECK)
    JL_VARIANTS_F64(JL_CHECK)
#undef JL_CHECK
    return false;
}

int variant_list(int precision, int32_t *pairs, int cap)
{
    int n = 0;
    // (0, 0): the static tile kernel
    if (pairs && n < cap) {
        pairs[0] = 0;
        pairs[1] = 0;
    }
    ++n;
    if (precision == JL_FP32)
        for (int t : {8, 16}) {
            if (pairs && n < cap) {
                pairs[2 * n] = 0;
                pairs[2 * n + 1] = t;
            }
            ++n;
        }
#define JL_LIST(T, P, UU)                                            \
    if ((sizeof(T) == 8) == (precision == JL_FP64)) {                \
        if (pairs && n < cap) { pairs[2 * n] = P; pairs[2 * n + 1] = UU; } \
        ++n;                                                         \
    }
    JL_VARIANTS_F32(JL_LIST)
    JL_VARIANTS_F64(JL_LIST)
#undef JL_LIST
    return n;
}

// Tile parts a warp claims per increment of the launch counter.  One part at a
// time balances best, but with thousands of parts per warp (large batches of
// low-count frames) the one counter becomes a hot spot: then up to 8 parts
// (one tile) per claim, keeping at least ~500 claims per warp.
static int32_t tile_claim(long long total_tiles, long long grid)
{
    const long long per_warp = (total_tiles * 8) / (grid * 8 > 0 ? grid * 8 : 1);
    int32_t c = 1;
    while (c < 8 && per_warp >= 1024LL * c)
        c *= 2;
    return c;
}

// Output specialisation of a launch: the batch plan's (computed over its
// frames), or that of the single frame.
static int launch_out_mode(const EscapeArgs &a)
{
    if (a.frames)
        return a.out_mode;
    const Frame &F = a.single;
    if (F.hist_bins || !F.rgba)
        return 0;
    if (!F.counts)
        return 2;
    return F.count_type == JL_COUNT_U16 ? 1 : F.count_type == JL_COUNT_U8 ? 3 : 0;
}

template <typename T>
static cudaError_t launch_static(const EscapeArgs &a, cudaStream_t st)
{
    size_t smem = 0;
    if (a.hist_smem && !a.frames)
        smem = (size_t)(a.single.max_iter + 1) * sizeof(uint32_t);
    auto kern = a.frames ? escape_static_kernel<T, true, 0> : escape_static_kernel<T, false, 0>;
    if constexpr (sizeof(T) == 4) {
        const int out_mode = launch_out_mode(a);
        if (out_mode == 1)
            kern = a.frames ? escape_static_kernel<T, true, 1> : escape_static_kernel<T, false, 1>;
        else if (out_mode == 2)
            kern = a.frames ? escape_static_kernel<T, true, 2> : escape_static_kernel<T, false, 2>;
        else if (out_mode == 3)
            kern = a.frames ? escape_static_kernel<T, true, 3> : escape_static_kernel<T, false, 3>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    if (a.total_tiles < 1)
        return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), 256, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    const int sms = device_sm_count();
    long long grid = (long long)(sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
    if (grid > a.total_tiles)
        grid = a.total_tiles;
    EscapeArgs b = a;
    b.claim = tile_claim(a.total_tiles, grid);
    kern<<<(unsigned)grid, 256, smem, st>>>(b);
    return cudaGetLastError();
}

static cudaError_t launch_compact(const EscapeArgs &a, int T, cudaStream_t st)
{
    size_t smem = 0;
    if (a.hist_smem && !a.frames)
        smem = (size_t)(a.single.max_iter + 1) * sizeof(uint32_t);
    // (the compacting kernel has the uint16 + RGBA8 specialisation only)
    const int out_mode = launch_out_mode(a);
    auto kern = a.frames ? (out_mode == 1 ? escape_compact_kernel<true, 8, 1> : escape_compact_kernel<true, 8, 0>)
                         : (out_mode == 1 ? escape_compact_kernel<false, 8, 1> : escape_compact_kernel<false, 8, 0>);
    if (smem > 16 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    if (a.total_tiles < 1)
        return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), 256, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    const int sms = device_sm_count();
    long long grid = (long long)(sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
    if (grid > a.total_tiles)
        grid = a.total_tiles;
    EscapeArgs b = a;
    b.claim = tile_claim(a.total_tiles, grid);
    kern<<<(unsigned)grid, 256, smem, st>>>(b, T);
    return cudaGetLastError();
}

// The certified binary32 pass of a binary64 launch (tile kernel).
static cudaError_t launch_cert(const EscapeArgs &a, cudaStream_t st)
{
    size_t smem = 0;
    if (a.hist_smem && !a.frames)
        smem = (size_t)(a.single.max_iter + 1) * sizeof(uint32_t);
    auto kern = a.frames ? cert_kernel<true, 0> : cert_kernel<false, 0>;
    if (launch_out_mode(a) == 1)
        kern = a.frames ? cert_kernel<true, 1> : cert_kernel<false, 1>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    if (a.total_tiles < 1)
        return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), 256, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    const int sms = device_sm_count();
    long long grid = (long long)(sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
    if (grid > a.total_tiles)
        grid = a.total_tiles;
    EscapeArgs b = a;
    b.claim = tile_claim(a.total_tiles, grid);
    kern<<<(unsigned)grid, 256, smem, st>>>(b);
    return cudaGetLastError();
}

// The double-float pass over the binary32 pass's list (persistent lane-refill
// kernel; the list's length is known only on the device).
static cudaError_t launch_cert2(const EscapeArgs &a, int num_sms, cudaStream_t st)
{
    size_t smem = 0;
    if (a.hist_smem && !a.frames)
        smem = (size_t)(a.single.max_iter + 1) * sizeof(uint32_t);
    auto kern = a.frames ? cert2_kernel<true, 0> : cert2_kernel<false, 0>;
    if (launch_out_mode(a) == 1)
        kern = a.frames ? cert2_kernel<true, 1> : cert2_kernel<false, 1>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), 256, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    const long long grid = (long long)(num_sms > 0 ? num_sms : 148) * (per_sm > 0 ? per_sm : 1);
    kern<<<(unsigned)grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

// Whether a binary64 launch with variant v takes the certified pass: a
// lane-refill variant, a list, the counters, and binary32 tables with tile
// tables (batches) or in the single frame.
static bool use_cert(const EscapeArgs &a, int precision, const Variant &v)
{
    if (precision != JL_FP64 || v.ppt == 0 || !a.cert_list || !a.cert_count || !a.list_counter)
        return false;
    return a.frames ? (a.tile_frame && a.tile_local)
                    : (a.single.xs32 && a.single.ys32 && a.single.xs32lo && a.single.ys32lo);
}

cudaError_t launch_escape(const EscapeArgs &a_in, int precision, const Variant &v, int num_sms, cudaStream_t st,
                          cudaEvent_t mid, cudaEvent_t mid2, cudaEvent_t done)
{
    EscapeArgs a = a_in;
    if (use_cert(a, precision, v)) {
        cudaError_t e = launch_cert(a, st);
        if (e == cudaSuccess && mid)
            e = cudaEventRecordWithFlags(mid, st, cudaEventRecordExternal);
        const bool two = a.cert_list2 && a.cert_count2 && a.list2_counter;
        if (e == cudaSuccess && two)
            e = launch_cert2(a, num_sms, st);
        if (e == cudaSuccess && mid2)
            e = cudaEventRecordWithFlags(mid2, st, cudaEventRecordExternal);
        if (e == cudaSuccess && done)
            e = cudaEventRecord(done, st);
        if (e != cudaSuccess)
            return e;
        EscapeArgs b = a;
        b.chunk_counter = a.list_counter;
        if (two) {
            // the binary64 kernel renders the double-float pass's list
            b.cert_list = a.cert_list2;
            b.cert_count = a.cert_count2;
        }
        const size_t smem = refill_smem_bytes(true, v.ppt, v.threads,
                                              (b.hist_smem && !b.frames) ? (size_t)b.single.max_iter + 1 : 0);
#define JL_DISPATCH_LIST(T, P, UU)                                                            \
        if (sizeof(T) == 8 && v.ppt == P && v.unroll == UU)                                   \
            return launch_one<T, P, UU, true>(b, v, num_sms, smem, st);
        JL_VARIANTS_F64(JL_DISPATCH_LIST)
#undef JL_DISPATCH_LIST
        return cudaErrorInvalidValue;
    }
    if (v.ppt == 0 && v.unroll > 0 && precision == JL_FP32)
        return launch_compact(a, v.unroll, st);
    if (v.ppt == 0)
        return precision == JL_FP64 ? launch_static<double>(a, st) : launch_static<float>(a, st);
    const size_t smem = refill_smem_bytes(precision == JL_FP64, v.ppt, v.threads,
                                          (a.hist_smem && !a.frames) ? (size_t)a.single.max_iter + 1 : 0);
#define JL_DISPATCH(T, P, UU)                                                                 \
    if (((sizeof(T) == 8) == (precision == JL_FP64)) && v.ppt == P && v.unroll == UU)         \
        return launch_one<T, P, UU>(a, v, num_sms, smem, st);
    JL_VARIANTS_F32(JL_DISPATCH)
    JL_VARIANTS_F64(JL_DISPATCH)
#undef JL_DISPATCH
    return cudaErrorInvalidValue;
}

Variant default_variant(int precision, int max_iter)
{
    (void)max_iter;
    if (precision == JL_FP64)
        // 4 pixels per lane in blocks of 8 steps: with the certified passes the
        // binary64 kernel renders long-lived pixels only (sweep list kernel
        // 3.59 ms with blocks of 4, 3.31 ms with blocks of 8)
        return Variant{4, 8, 128, 0};
    // binary32: the compacting tile kernel, parking threshold 16 (ahead of the
    // lane-refill kernel on every sweep frame; within a few % of the static
    // kernel on frames that escape early, far ahead on divergent ones)
    return Variant{0, 16, 256, 0};
}

}  // namespace jl
