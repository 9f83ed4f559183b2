/*
 * jl.h — C ABI of libjl.so, a B300 (sm_103a) escape-time fractal renderer and
 * parameter-space surveyor.
 *
 * The method is the escape-time algorithm of "Fractal Art Generation using
 * GPUs" (arXiv:1611.03079):
 *   Sec. 2  region covering: pixel (i, j) of a W x H grid is mapped to a point
 *           of a rectangle of the complex plane; Z_{n+1} = Z_n^2 + C is
 *           iterated from that point up to an iteration limit (100 in the
 *           paper) and the pixel is coloured by the number of iterations
 *           taken to escape;
 *   Sec. 3  Mandelbrot (parameter-plane) mode: Z_0 = 0 and C = pixel; deep
 *           zooms that need extra precision; paths of C for animation.
 *
 * Conventions shared by every entry point
 *   - Pixel centres.  dx = (xmax - xmin) / W and dy = (ymax - ymin) / H in
 *     binary64; pixel (i, j) is x = xmin + (i + 0.5) dx, y = ymin + (j + 0.5) dy,
 *     evaluated in binary64 without fused multiply-add and then rounded once
 *     (round-to-nearest-even) to the working precision.  Row j = 0 is y = ymin;
 *     images are row-major with pitch W.
 *   - Iteration.  With (x, y) = Z and (cr, ci) = C in the working precision,
 *     each step is: x2 = x*x; y2 = y*y; escape if x2 + y2 > 4; y = (x + x)*y + ci;
 *     x = (x2 - y2) + cr; every operation rounded to nearest, none fused.
 *     C given in binary64 is rounded once to the working precision.
 *   - Count.  The number of updates made before the first failing test; 0 if
 *     |Z_0|^2 > 4; max_iter if no test among n = 0 .. max_iter-1 fails.
 *   - Colour (Sec. 2 colour levels).  count == max_iter -> palette entry 255;
 *     otherwise entry (count * 255) / max_iter (unsigned integer division).
 *     The palette is 256 RGBA8 entries (1024 bytes, R first).
 *   - Histogram.  hist[b] = #{pixels with count b} / (W*H), b = 0 .. max_iter,
 *     the quotient formed in binary64 and rounded once to binary32.
 *   - Memory.  Unless stated otherwise, output pointers are caller-owned device
 *     memory; the library allocates only stream-ordered scratch
 *     (cudaMallocAsync on the caller's stream) and frees it on that stream.
 *   - Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless stated otherwise.
 *   - Errors.  Every function returns a jl_status.  No exception crosses the
 *     ABI.  jl_last_error() returns a thread-local message for the last
 *     failure on the calling thread.  Argument errors are detected on the host
 *     before anything is launched; JL_ECUDA reports a failed CUDA call.
 */
#ifndef JL_H
#define JL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JL_OK = 0,
    JL_EINVAL = 1,       /* invalid argument (checked on the host) */
    JL_ECUDA = 2,        /* a CUDA runtime call failed */
    JL_ENOMEM = 3,       /* device or host allocation failed */
    JL_ETIMEOUT = 4,     /* a launch exceeded its cycle budget and stopped early */
    JL_EUNSUPPORTED = 5  /* no usable sm_103a device */
} jl_status;

typedef enum { JL_FP32 = 0, JL_FP64 = 1, JL_AUTO = 2 } jl_precision;
typedef enum { JL_JULIA = 0, JL_MANDELBROT = 1 } jl_mode;
typedef enum { JL_COUNT_NONE = 0, JL_COUNT_U8 = 1, JL_COUNT_U16 = 2 } jl_count_type;

/* Axis-aligned rectangle of the complex plane (Sec. 2 region covering).
 * Requires finite values with xmin < xmax and ymin < ymax. */
typedef struct {
    double xmin, xmax, ymin, ymax;
} jl_rect;

/* Thread-local text of the last error on the calling thread ("" if none). */
const char *jl_last_error(void);

/* Library version string. */
const char *jl_version(void);

/*
 * Precision rule for deep zooms (Sec. 3: deep zooms need extra precision).
 * Returns JL_FP64 when min(dx, dy) < 1000 * ulp32(m), m being the largest of
 * |xmin|, |xmax|, |ymin|, |ymax| rounded to binary32 and ulp32(m) the gap from
 * m to the next larger binary32 value; otherwise JL_FP32.  Returns -1 on an
 * invalid rectangle or size.  Host-only, no GPU needed.
 */
int jl_select_precision(jl_rect rect, int32_t width, int32_t height);

/*
 * Render one frame (Sec. 2; Sec. 3 for JL_MANDELBROT and deep zoom).
 *   cr, ci      C for JL_JULIA (ignored for JL_MANDELBROT), binary64
 *   rect        view, see jl_rect
 *   width, height  1 .. 65536 each, width*height < 2^31
 *   max_iter    iteration limit, 1 .. 65535 (the paper uses 100)
 *   precision   JL_FP32, JL_FP64, or JL_AUTO (jl_select_precision)
 *   mode        JL_JULIA (Z_0 = pixel) or JL_MANDELBROT (Z_0 = 0, C = pixel)
 *   count_type  JL_COUNT_U8 (requires max_iter <= 255), JL_COUNT_U16, or
 *               JL_COUNT_NONE (counts must then be NULL)
 *   counts      device, width*height elements of count_type, or NULL
 *   rgba        device, width*height*4 bytes, or NULL
 *   palette     HOST pointer to 1024 bytes (256 RGBA8 entries) or NULL for
 *               the built-in palette (see jl_default_palette); read before
 *               the call returns
 *   hist        device, max_iter + 1 floats, or NULL; the buffer is used as
 *               uint32 bin storage during the call and holds the normalised
 *               histogram when the stream reaches the end of the call
 *   stream      cudaStream_t
 * At least one of counts, rgba, hist must be non-NULL.  The call takes
 * stream-ordered device scratch (cudaMallocAsync, freed in stream order):
 * the coordinate tables, and for binary64 frames their float-pair roundings
 * and the two lists of the certified passes (16 bytes per pixel): a binary32
 * and then a float-pair orbit, each with a rigorous bound on its distance to
 * the binary64 orbit, settle the pixels whose every binary64 escape test the
 * bound decides; the rest are iterated in binary64.  The counts are the
 * binary64 counts either way (jl_render_static allocates nothing and iterates
 * every binary64 pixel in binary64).
 */
int jl_render(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
              int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
              const uint8_t *palette, float *hist, void *stream);

/*
 * Same as jl_render but every output pointer is HOST memory (pinned or
 * pageable).  The frame is rendered into stream-ordered device scratch and
 * copied back; the call returns after the copies complete (it synchronises
 * `stream`).  Used for end-to-end measurements that include the transfers.
 */
int jl_render_to_host(double cr, double ci, jl_rect rect, int32_t width, int32_t height,
                      int32_t max_iter, int32_t precision, int32_t mode, int32_t count_type,
                      void *counts_host, uint8_t *rgba_host, const uint8_t *palette,
                      float *hist_host, void *stream);

/*
 * jl_render with an explicit kernel variant (used by the autotuner and the
 * tests): ppt independent pixels per thread, unroll steps between service
 * points, threads per CTA (multiple of 32, 32..256), ctas_per_sm (0 = the
 * occupancy maximum).  ppt = unroll = 0 selects the static kernel (one pixel
 * per thread, 32 x 32 pixel tiles taken by warps in 8 x 16 parts; threads and
 * ctas_per_sm are then ignored).  ppt = 0 with unroll = T in 1..32 (binary32
 * only) selects the compacting tile kernel: the static kernel's tiles, with a
 * patch's live pixels parked in a per-warp ring once T or fewer of its 32
 * are left and resumed later as full batches of 32.  Unsupported (ppt, unroll) pairs return JL_EINVAL;
 * jl_variant_list() enumerates the supported ones.
 */
int jl_render_variant(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
                      int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
                      const uint8_t *palette, float *hist, int32_t ppt, int32_t unroll, int32_t threads,
                      int32_t ctas_per_sm, void *stream);

/*
 * Writes up to `cap` supported (ppt, unroll) pairs for `precision` into
 * `pairs` (2 ints each) and returns how many exist (may exceed cap), or -1
 * for an invalid precision.
 */
int jl_variant_list(int32_t precision, int32_t *pairs, int32_t cap);

/*
 * Issue-rate probe, the denominator of the escape kernels' ALU roofline.
 * kind 0 (JL_FP32) / 1 (JL_FP64): 8 independent multiply/add chains per
 * thread, 8 CTAs of 256 threads on every SM (separate FMUL and FADD, DMUL
 * and DADD, no FMA); kind 2: packed binary32 pairs, separate chains of
 * add.rn.f32x2 and mul.rn.f32x2 (two lane operations per instruction; no
 * product feeds a sum).  Returns the achieved lane operations per second in
 * *lane_ops_per_s (and the kernel time in *seconds if non-NULL); JL_EINVAL
 * for another kind.  Synchronises `stream`.
 */
int jl_probe_peak(int32_t kind, int32_t iters, double *lane_ops_per_s, double *seconds, void *stream);

/*
 * Size of the static scratch array used by jl_render_static (bytes).
 */
#define JL_STATIC_SCRATCH_BYTES (256u * 1024u)

/*
 * jl_render_static — jl_render without any device allocation.  The paper has
 * no counterpart; this entry point exists for callers that cannot allocate
 * device memory when they render: a real-time display loop that must not
 * stall on an allocation (cudaMalloc can synchronise the whole device), or a
 * process whose device memory is reserved up front by another allocator (for
 * example a framework's caching allocator), where any further allocation
 * fails or fragments that reservation.
 *
 * Arguments, outputs and results are those of jl_render (counts, rgba and
 * hist are caller-owned device buffers; palette is a host pointer or NULL),
 * and so is the kernel: the autotuned variant when jl_autotune has run or a
 * tuning table was loaded, else the default one.  Binary64 frames skip the
 * certified passes (they need per-pixel lists): every pixel is iterated in
 * binary64, with the same counts.
 * The scratch it needs (coordinate tables, work counter, status word) lives
 * in one file-scope device array of JL_STATIC_SCRATCH_BYTES bytes, which
 * every GPU that loads the library holds until the process exits.
 *   - Limit: (width + height) * 4 bytes (binary32) or * 8 bytes (binary64),
 *     rounded up to 256, plus 256 must fit in JL_STATIC_SCRATCH_BYTES, i.e.
 *     width + height <= 65472 in binary32 and <= 32736 in binary64.  Larger
 *     frames return JL_EINVAL with the limit in jl_last_error().
 *   - Set-up: the first call on a device (with that device current) looks up
 *     the array's device address with cudaGetSymbolAddress and keeps it for
 *     the life of the process; make that first call before any stream
 *     capture.  cudaDeviceReset destroys the module that holds the array, so
 *     the kept address is stale afterwards: do not call this entry point
 *     after resetting the device.
 *   - Sharing: every call on a device uses the same array and leaves its
 *     contents behind; each call clears the counter and status it relies on
 *     (with cudaMemsetAsync, which does not allocate).  Calls whose work
 *     overlaps on the GPU (concurrent streams, or host threads issuing to
 *     different streams) race on the array: serialise them on one stream.
 *   - It calls no cudaMalloc, cudaMallocAsync, cudaFree or other allocating
 *     routine.
 */
int jl_render_static(double cr, double ci, jl_rect rect, int32_t width, int32_t height, int32_t max_iter,
                     int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
                     const uint8_t *palette, float *hist, void *stream);

/* ------------------------------------------------------------------------
 * Generic maps (Sec. 2: many other functions than Z^2 + C give fractal
 * images; Fig. 4: a rational map with C = .862085 + .64695i; Sec. 5: freer
 * functional forms).  Two families, iterated as Z <- F(Z) + C:
 *   JL_MAP_POWER     F(Z) = Z^d, 2 <= d <= 16;
 *   JL_MAP_RATIONAL  F(Z) = P(Z) / Q(Z), P and Q of degree 0..8 with complex
 *                    coefficients (Fig. 4's formula as printed is one case).
 * Step, in the working precision, every operation rounded to nearest and
 * none fused: x2 = x*x; y2 = y*y; escape unless x2 + y2 <= bailout (a NaN
 * escapes); (fx, fy) = F(x, y); x = fx + cr; y = fy + ci.
 *   Z^d: W = Z, then for each bit of d below the leading one, from high to
 *     low: W = (a*a - b*b, (a + a)*b) for W = (a, b), and, when the bit is
 *     set, W = (a*x - b*y, a*y + b*x).  d = 2 reproduces the quadratic
 *     iteration of the other entry points bit for bit.
 *   P(Z): Horner from the leading coefficient, P = P*Z + a_k with the
 *     product formed as above; P/Q = ((pr*qr + pi*qi) / (qr*qr + qi*qi),
 *     (pi*qr - pr*qi) / (qr*qr + qi*qi)) with correctly rounded division.
 * Coefficients, bailout and z0 are given in binary64 and rounded once to the
 * working precision.  Count, colour, histogram, pixel centres and precision
 * selection are those of jl_render.
 * ------------------------------------------------------------------------ */
typedef enum { JL_MAP_POWER = 0, JL_MAP_RATIONAL = 1 } jl_map_kind;

typedef struct {
    int32_t kind;        /* jl_map_kind */
    int32_t degree;      /* JL_MAP_POWER: d, 2..16 */
    int32_t num_degree;  /* JL_MAP_RATIONAL: degree of P, 0..8 */
    int32_t den_degree;  /* JL_MAP_RATIONAL: degree of Q, 0..8 */
    double num[18];      /* P: (re, im) pairs, constant term first; unused entries ignored */
    double den[18];      /* Q: (re, im) pairs, constant term first */
    double bailout;      /* escape radius squared, > 0 and finite (4 for radius 2) */
    double z0r, z0i;     /* JL_MANDELBROT mode: Z_0 (usually a critical point of F; 0 for Z^d) */
} jl_map;

/* Render one frame of a generic map.  Arguments after `map` as jl_render
 * (mode JL_JULIA: Z_0 = pixel, C = (cr, ci); JL_MANDELBROT: Z_0 = (z0r, z0i),
 * C = pixel).  `map` is a host pointer read during the call only.
 * JL_EINVAL for a NULL map, an unknown kind, a degree out of range, a
 * non-finite coefficient, bailout or z0, or any jl_render argument error. */
int jl_render_map(const jl_map *map, double cr, double ci, jl_rect rect, int32_t width, int32_t height,
                  int32_t max_iter, int32_t precision, int32_t mode, int32_t count_type, void *counts, uint8_t *rgba,
                  const uint8_t *palette, float *hist, void *stream);

/* ------------------------------------------------------------------------
 * Batches (Sec. 3: paths of C rendered as animations; also the histogram
 * targets of the surrogate).  A plan renders many frames -- each with its own
 * C, view, size, limit, mode and precision -- in one CUDA-graph launch of
 * persistent escape kernels.
 * ------------------------------------------------------------------------ */

/* One frame of a batch.  Offsets are in bytes from the base pointers given to
 * jl_batch_create; -1 means "no such output".  rgba and hist offsets must be
 * multiples of 4, uint16 counts offsets multiples of 2. */
typedef struct {
    double cr, ci;          /* C for JL_JULIA frames */
    jl_rect rect;
    int32_t width, height, max_iter;
    int32_t mode;           /* JL_JULIA / JL_MANDELBROT */
    int32_t precision;      /* JL_FP32 / JL_FP64 / JL_AUTO (jl_select_precision) */
    int32_t count_type;     /* JL_COUNT_*; must be JL_COUNT_NONE when counts_offset < 0 */
    int64_t counts_offset;
    int64_t rgba_offset;
    int64_t hist_offset;    /* max_iter + 1 floats at this offset */
} jl_frame;

/* Plan options; zero-initialise for defaults. */
typedef struct {
    int32_t chunk_len;      /* pixels per work chunk, 16..1024; 0 = 512 */
    int32_t fp32_ppt, fp32_unroll, fp32_threads;  /* all 0 = tuned or default variant */
    int32_t fp64_ppt, fp64_unroll, fp64_threads;
    int32_t variant_flags;  /* bit 0 / bit 1: the fp32 / fp64 (ppt, unroll) pair is given explicitly
                               (needed for the static kernel, ppt = unroll = 0);
                               bit 2: no certified binary32 pass for binary64 frames (every binary64
                               pixel then runs on the binary64 kernel; for comparisons);
                               bit 3: record timing events around the kernels inside the graph
                               (jl_batch_phase_ms);
                               bit 4: no double-float pass after the binary32 one (the binary64
                               kernel renders every pixel the binary32 pass lists) */
    int32_t tune;           /* 1: for each precision group without an explicit variant, time
                               candidate kernels (the tuned and the default variant, the tile
                               kernels, a few lane-refill shapes for binary64) on the plan's own
                               frames at creation and keep the fastest; 0: the tuned or default
                               variant */
    int64_t cycle_budget;   /* per-CTA clock64 budget; when exceeded the kernels stop
                               taking work and the plan status becomes JL_ETIMEOUT;
                               0 = unlimited */
} jl_batch_opts;

typedef struct jl_batch jl_batch;

/*
 * Build a plan for n frames writing to counts_base / rgba_base / hist_base
 * (device memory, caller-owned, bound to the plan).  Allocates the plan's
 * tables, computes every coordinate table, and captures the launch graph;
 * synchronous.  palette: host, 1024 bytes, or NULL for the built-in one.
 * On success *out owns device memory until jl_batch_destroy.
 */
int jl_batch_create(const jl_frame *frames, int32_t n, void *counts_base, uint8_t *rgba_base, float *hist_base,
                    const uint8_t *palette, const jl_batch_opts *opts, jl_batch **out);

/* The kernel variant the plan uses for a precision group (chosen at creation:
 * explicit option, the plan's own timing with opts.tune, else the tuned or
 * default one); meaningful for groups that have frames. */
int jl_batch_variant(const jl_batch *b, int32_t precision, int32_t *ppt, int32_t *unroll, int32_t *threads);

/* Render every frame of the plan: one cudaGraphLaunch on `stream`
 * (asynchronous; nothing is allocated). */
int jl_batch_launch(jl_batch *b, void *stream);

/* Status word of the last launch (JL_OK or JL_ETIMEOUT); synchronises `stream`. */
int jl_batch_status(jl_batch *b, void *stream, int32_t *status_out);

/* Resolved precision of each frame (input order) into out[0..cap); returns n, or -1. */
int jl_batch_precisions(const jl_batch *b, int32_t *out, int32_t cap);

/* Pixel totals of the binary32 and binary64 frames of the plan. */
int jl_batch_pixels(const jl_batch *b, int64_t *fp32_pixels, int64_t *fp64_pixels);

/* Counters of the last launch's binary64 frames, into out[0..5]: the pixels
 * the certified binary32 pass left unsettled; the pixels left to the binary64
 * kernel after the double-float pass (equal to out[0] when that pass is off);
 * the iterations (sum of counts) of the pixels the double-float pass settled;
 * the iterations the binary64 kernel ran; the tests (steps) the binary32 pass
 * and the double-float pass decided (each pixel's tests up to its escape, its
 * limit or its unsettled test).  Zeros when the plan has no binary64 frames or
 * the passes are off.  Synchronises `stream`.  The certified passes
 * run a binary32 (then double-float) orbit with a rigorous bound on its
 * distance to the binary64 orbit and keep a pixel only when the bound settles
 * every binary64 test of the pixel (the counts are the binary64 counts either
 * way; paper Sec. 3, precision of deep zooms). */
int jl_batch_cert_stats(jl_batch *b, void *stream, int64_t *out);

/* Device time (ms) of the phases of the last completed launch of a plan
 * created with opts.variant_flags bit 3 (timing events recorded inside its
 * graph): ms_out[0] the binary32 escape kernel, ms_out[1] the certified
 * binary32 pass of the binary64 frames, ms_out[2] the double-float pass,
 * ms_out[3] the binary64 escape kernel; -1 for a phase the plan does not run.
 * The launch must have completed (synchronise its stream first).  JL_EINVAL
 * without the flag. */
int jl_batch_phase_ms(const jl_batch *b, float *ms_out);

/* Frees the plan (after its launches have completed). */
void jl_batch_destroy(jl_batch *b);

/* One-shot: create, launch, wait, destroy.  Synchronous; returns JL_ETIMEOUT
 * never (no budget) and JL_OK on success. */
int jl_render_batch(const jl_frame *frames, int32_t n, void *counts_base, uint8_t *rgba_base, float *hist_base,
                    const uint8_t *palette, void *stream);

/*
 * Render n frames into HOST memory with the device-to-host copies overlapped
 * with rendering.  Frames as in jl_batch_create (offsets in bytes from the
 * host base pointers, -1 = no such output; counts_host / rgba_host /
 * hist_host may be NULL when no frame uses them).  Renders and copies run
 * on separate internal streams (up to 4 render and 2 copy streams): frame i
 * renders into device slot i mod depth and is copied out as soon as its
 * render is done, while later frames render; a render waits for a copy only
 * to reuse a slot; the last frame may render as row bands copied band by
 * band (see jl_host_plan_launches).  `depth` = device slots, 1..64, or 0 for
 * the default (one slot per frame up to 16 frames, at most 4 GiB of slots).  The host buffers
 * should be pinned (page-locked) for the copies to overlap; pageable memory
 * works but serialises.  Work queued earlier on `stream` is waited for; the
 * call returns when every copy has completed (synchronous).  The library
 * allocates `depth` slots of the largest frame's outputs for the duration of
 * the call.  Errors: as jl_batch_create for the frame descriptions;
 * JL_EINVAL for a depth outside 0..64; JL_ECUDA / JL_ENOMEM from the device.
 */
int jl_render_frames_to_host(const jl_frame *frames, int32_t n, void *counts_host, uint8_t *rgba_host,
                             float *hist_host, const uint8_t *palette, int32_t depth, void *stream);

/*
 * The same as a reusable plan: jl_host_plan_create validates the frames and
 * does the once-per-frame-set work (`depth` device slots, room for the
 * coordinate tables, internal streams and events); every jl_host_plan_run
 * computes each frame's coordinate tables from its description (the region
 * covering of Sec. 2) and renders every frame into the host buffers given at
 * creation (which must stay valid while the plan lives), with the copies
 * overlapped, and returns when the last copy has completed.  Runs on the device current at creation (JL_EINVAL otherwise).
 * The palette (1024 bytes, or NULL for the default) is copied at creation.
 * jl_host_plan_destroy waits for outstanding work and frees everything.
 */
typedef struct jl_host_plan jl_host_plan;
int jl_host_plan_create(const jl_frame *frames, int32_t n, void *counts_host, uint8_t *rgba_host, float *hist_host,
                        const uint8_t *palette, int32_t depth, jl_host_plan **out);
int jl_host_plan_run(jl_host_plan *plan, void *stream);
void jl_host_plan_destroy(jl_host_plan *plan);
/* Escape-kernel launches per run: one per frame, plus the row bands of the
 * last frame (a last frame without a histogram whose counts + RGBA reach
 * 8 MB renders as bands of about 8 MB, at most 4, each a multiple of 32 rows,
 * copied out band by band).  -1 for a NULL plan. */
int32_t jl_host_plan_launches(const jl_host_plan *plan);

/* ------------------------------------------------------------------------
 * Autotuner of the escape kernel's launch shape.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t ppt, unroll, threads, ctas_per_sm;
    double ms;              /* mean time of the calibration set with this variant */
    int32_t candidates;     /* candidates timed (jl_tune_get: 1 if tuned, 0 if default) */
} jl_tune_result;

/*
 * Times every supported (ppt, unroll) x {128, 256} threads on the calibration
 * frames (their own rect, size, mode and C; `precision` and `max_iter` as
 * given), `reps` timed repetitions each after one warm-up, and records the
 * fastest for (current device, precision, bucket of max_iter: <=128, <=1024,
 * <=8192, larger).  calib may be NULL (built-in set: a 1024^2 Julia frame and
 * a 1024^2 Mandelbrot frame).  jl_render and new batch plans use the
 * recorded variant.  Synchronous.
 */
int jl_autotune(int32_t precision, int32_t max_iter, const jl_frame *calib, int32_t n_calib, int32_t reps,
                jl_tune_result *out);

/* The variant jl_render would use now for (precision, max_iter). */
int jl_tune_get(int32_t precision, int32_t max_iter, jl_tune_result *out);

/* Forget all tuned variants (back to the defaults). */
int jl_tune_clear(void);

/* Save / load the tuning table (text, one entry per line). */
int jl_tune_save(const char *path);
int jl_tune_load(const char *path);

/* ------------------------------------------------------------------------
 * Learned screening surrogate (the paper's aim of sampling the parameter
 * space quickly, Sec. 1, with the Mandelbrot set as the roadmap for C,
 * Sec. 3).  A fixed network maps C to the normalised escape-count histogram of
 * its Julia frame (128 x 128 over [-2,2]^2, limit 100):
 *   phi(C) = [sin(2 pi B C), cos(2 pi B C)] with B (32 x 2, row-major) fixed,
 *   h1 = relu(phi W1^T + b1) (64 -> 256), h2 = relu(h1 W2^T + b2) (256 -> 256),
 *   p = softmax(h2 W3^T + b3) (256 -> 101);
 * bfloat16 weights and activations in every matrix product, binary32
 * accumulation (tcgen05 tensor cores), cross-entropy loss, Adam on binary32
 * master weights.  Parameter block order (binary32, jl_model_num_params()
 * values): W1[256x64] b1[256] W2[256x256] b2[256] W3[101x256] b3[101], W
 * row-major (out x in).  All C arrays are device memory, n x 2 binary32
 * (real, imaginary); histograms are n x 101 binary32.
 * ------------------------------------------------------------------------ */
typedef struct jl_model jl_model;

/* Number of binary32 values in the parameter block (108389). */
int jl_model_num_params(void);

/* Creates a model on the current device from host arrays: fourier_B (64
 * floats) and init_params (jl_model_num_params() floats); Adam state zero. */
int jl_model_create(const float *fourier_B, const float *init_params, jl_model **out);
void jl_model_destroy(jl_model *md);

/* Copies parameters / Adam moments / step between host and device (NULL
 * pointers are skipped).  Synchronous. */
int jl_model_get_state(const jl_model *md, float *params, float *m, float *v, int32_t *step);
int jl_model_set_state(jl_model *md, const float *params, const float *m, const float *v, const int32_t *step);

/* Forward pass over n values of C: probs (n x 101) and/or score (n, the
 * entropy of the predicted histogram in nats), either may be NULL.  One
 * persistent fused kernel (features, three tensor-core products, softmax)
 * with activations kept on chip.  Asynchronous on `stream`. */
int jl_model_forward(jl_model *md, const float *c, int64_t n, float *probs, float *score, void *stream);

/* The same forward built from one launch of the general tensor-core product
 * kernel per layer; a reference for jl_model_forward's fused kernel. */
int jl_model_forward_layered(jl_model *md, const float *c, int64_t n, float *probs, float *score, void *stream);

/* Loss and gradients (host outputs, NULL skipped) of one batch of n <= 65536
 * rows against target histograms; no parameter update.  One launch of the
 * fused training-step kernel (forward, softmax error and backward of every
 * 128-row tile, per-tile partials) and a fixed-order sum of the partials.
 * Synchronous. */
int jl_model_grads(jl_model *md, const float *c, const float *target, int32_t n, float *loss_host, float *grads_host,
                   void *stream);

/* Adam training: `epochs` passes over n samples in batches of `batch` (the
 * last partial batch of each pass is dropped).  order: device, epochs x n
 * sample indices (one permutation per pass, chosen by the caller), or NULL
 * to take samples in order.  The learning rate follows a cosine from lr at
 * the first step of the call to lr_final after the last (lr_final == lr:
 * constant).  loss_curve: host, `epochs` mean batch losses, or NULL.  Each
 * step is two launches: the fused training-step kernel and Adam (which sums
 * the per-tile partials in a fixed order, so a resumed run continues bit for
 * bit).  Synchronous. */
int jl_train(jl_model *md, const float *c, const float *hist, int32_t n, const int32_t *order, int32_t epochs,
             int32_t batch, float lr, float lr_final, float *loss_curve, void *stream);

/* Top-k of n non-negative scores (device), ties broken by the smaller index,
 * descending: out_idx (k int32) and out_score (k floats, may be NULL).
 * 1 <= k <= min(n, 16384).  Allocates stream-ordered scratch. */
int jl_topk(const float *score, int64_t n, int32_t k, int32_t *out_idx, float *out_score, void *stream);

/* Screening: forward over n values of C (score = entropy of the predicted
 * histogram, written to `score`, n floats), then the top k by score
 * (1 <= k <= min(n, 16384)).  When a call has the same (c, n, k, output)
 * pointers as the previous call on the model, its work is captured as a CUDA
 * graph and replayed by later such calls (one graph launch instead of about
 * a dozen kernel launches); weights updated by training are picked up (the
 * graph reads the packed weight images, which every update rewrites in
 * place).  On a stream that is itself being captured, the launches are
 * issued directly.  Calls on one model must not overlap in time. */
int jl_survey(jl_model *md, const float *c, int64_t n, int32_t k, int32_t *top_idx, float *top_score, float *score,
              void *stream);

/* Per-row L1 distance of two histogram arrays (device): out[i] = sum_b |p - q|. */
int jl_hist_l1(const float *p, int32_t ldp, const float *q, int32_t ldq, int32_t n, int32_t bins, float *out,
               void *stream);

/* Checkpoint (parameters, Adam moments, step, Fourier matrix) to a
 * little-endian binary file, and back.  Resuming continues bit-identically. */
int jl_model_save(const jl_model *md, const char *path);
int jl_model_load(const char *path, jl_model **out);

/*
 * The tensor-core product on its own: C[M x N] (binary32, row stride ldc) =
 * A[M x K] * B[K x N] with bfloat16 operands (device).  a_trans = 0: A is
 * row-major M x K (A[m*lda + k]); 1: A is stored K x M (A[k*lda + m]).
 * b_trans = 0: B is stored N x K (B[n*ldb + k]); 1: B is stored K x N
 * (B[k*ldb + n]).  1 <= N <= 256.  status: device int32 set to JL_ETIMEOUT if
 * a wait gave up, or NULL.
 */
int jl_gemm_bf16(const void *A, int32_t lda, int32_t a_trans, const void *B, int32_t ldb, int32_t b_trans, int32_t M,
                 int32_t N, int32_t K, float *C, int32_t ldc, int32_t *status, void *stream);

/* Self-test of the integer-pipe doubling the binary64 kernels use for x + x:
 * out[i] = 2 * in[i] for n device doubles, computed exactly as the kernels do
 * (bit-identical to IEEE x + x except for NaN payloads). */
int jl_selftest_double(const double *in, double *out, int32_t n, void *stream);

/* Writes the built-in 256-entry RGBA8 palette (1024 bytes) to `out` (host).
 * Entry 255 (never-escaped points) is opaque black. */
int jl_default_palette(uint8_t *out);

#ifdef __cplusplus
}
#endif

#endif /* JL_H */
