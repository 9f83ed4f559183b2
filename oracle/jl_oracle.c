/*
 * CPU oracle for escape-time rendering (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The product path (libjl.so) never links or calls
 * it, and this file shares no code, header or table with the CUDA sources.
 *
 * What it computes (paper: "Fractal Art Generation using GPUs", Sec. 2 and 3):
 *   - region covering (Sec. 2): pixel (i, j) of a W x H grid maps to the pixel
 *     centre x_i = xmin + (i + 0.5) dx, y_j = ymin + (j + 0.5) dy with
 *     dx = (xmax - xmin) / W, dy = (ymax - ymin) / H, evaluated in binary64 and
 *     then rounded once to the working precision;
 *   - escape time for Z_{n+1} = Z_n^2 + C (Sec. 2) with an iteration limit
 *     (100 in the paper): the count is the number of updates made before the
 *     first failing test |Z|^2 > 4, or the limit when no test fails;
 *   - Mandelbrot (parameter-plane) mode (Sec. 3): Z_0 = 0 and C = pixel;
 *   - colour levels from the count (Sec. 2): a 256-entry RGBA8 palette,
 *     entry 255 for points that never escaped, else (count * 255) / limit;
 *   - the normalised escape-count histogram (bins 0..limit).
 * The iteration is written one IEEE operation per statement, in this order:
 *   x2 = x*x; y2 = y*y; escape if x2 + y2 > 4; t = x + x; t = t*y; y = t + ci;
 *   u = x2 - y2; x = u + cr.
 * Build flags (see oracle/build.py): -O2 -ffp-contract=off, no fast-math, so
 * every statement is one correctly rounded binary32/binary64 operation and no
 * multiply is fused with an add.  Subnormals are kept (default MXCSR).
 */
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define JLO_OK 0
#define JLO_EINVAL 1

/* Escape count of one point in binary32 (Sec. 2 escape-time rule). */
static int32_t escape_f32(float x, float y, float cr, float ci, int32_t max_iter)
{
    for (int32_t n = 0; n < max_iter; ++n) {
        float x2 = x * x;
        float y2 = y * y;
        float r = x2 + y2;
        if (r > 4.0f)
            return n;
        float t = x + x;
        t = t * y;
        y = t + ci;
        float u = x2 - y2;
        x = u + cr;
    }
    return max_iter;
}

/* Same rule in binary64 (deep zoom, Sec. 3). */
static int32_t escape_f64(double x, double y, double cr, double ci, int32_t max_iter)
{
    for (int32_t n = 0; n < max_iter; ++n) {
        double x2 = x * x;
        double y2 = y * y;
        double r = x2 + y2;
        if (r > 4.0)
            return n;
        double t = x + x;
        t = t * y;
        y = t + ci;
        double u = x2 - y2;
        x = u + cr;
    }
    return max_iter;
}

typedef struct {
    double cr, ci, xmin, xmax, ymin, ymax;
    int32_t W, H, max_iter, mode, precision;
    int32_t row0, row1;
    int32_t out_row_base;  /* row that maps to counts[0] */
    uint16_t *counts;
} job_t;

/* Region covering (Sec. 2) and the per-pixel loop of the sequential version. */
static void render_rows(const job_t *jb)
{
    const double dx = (jb->xmax - jb->xmin) / (double)jb->W;
    const double dy = (jb->ymax - jb->ymin) / (double)jb->H;
    for (int32_t j = jb->row0; j < jb->row1; ++j) {
        double yd = jb->ymin + ((double)j + 0.5) * dy;
        for (int32_t i = 0; i < jb->W; ++i) {
            double xd = jb->xmin + ((double)i + 0.5) * dx;
            int32_t n;
            if (jb->precision == 0) {
                float px = (float)xd, py = (float)yd;
                if (jb->mode == 0)
                    n = escape_f32(px, py, (float)jb->cr, (float)jb->ci, jb->max_iter);
                else
                    n = escape_f32(0.0f, 0.0f, px, py, jb->max_iter);
            } else {
                if (jb->mode == 0)
                    n = escape_f64(xd, yd, jb->cr, jb->ci, jb->max_iter);
                else
                    n = escape_f64(0.0, 0.0, xd, yd, jb->max_iter);
            }
            jb->counts[(size_t)(j - jb->out_row_base) * (size_t)jb->W + (size_t)i] = (uint16_t)n;
        }
    }
}

static void *render_thread(void *arg)
{
    render_rows((const job_t *)arg);
    return NULL;
}

/*
 * Escape counts of a W x H grid, row-major, row 0 at y = ymin.
 *   mode: 0 = Julia (Z_0 = pixel, C = (cr, ci)); 1 = Mandelbrot (Z_0 = 0, C = pixel)
 *   precision: 0 = binary32, 1 = binary64
 *   counts: host, W*H uint16 (caller-owned)
 *   nthreads: rows are split into contiguous bands, one per POSIX thread
 * Returns 0, or 1 on invalid arguments.
 */
int jlo_render(double cr, double ci, double xmin, double xmax, double ymin, double ymax,
               int32_t W, int32_t H, int32_t max_iter, int32_t mode, int32_t precision,
               uint16_t *counts, int32_t nthreads)
{
    if (W < 1 || H < 1 || max_iter < 1 || max_iter > 65535 || !counts)
        return JLO_EINVAL;
    if (mode != 0 && mode != 1)
        return JLO_EINVAL;
    if (precision != 0 && precision != 1)
        return JLO_EINVAL;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > H)
        nthreads = H;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return JLO_EINVAL;
    }
    for (int32_t k = 0; k < nthreads; ++k) {
        job_t *jb = &jobs[k];
        jb->cr = cr; jb->ci = ci;
        jb->xmin = xmin; jb->xmax = xmax; jb->ymin = ymin; jb->ymax = ymax;
        jb->W = W; jb->H = H; jb->max_iter = max_iter; jb->mode = mode;
        jb->precision = precision;
        jb->row0 = (int32_t)(((int64_t)H * k) / nthreads);
        jb->row1 = (int32_t)(((int64_t)H * (k + 1)) / nthreads);
        jb->out_row_base = 0;
        jb->counts = counts;
    }
    if (nthreads == 1) {
        render_rows(&jobs[0]);
    } else {
        for (int32_t k = 0; k < nthreads; ++k)
            pthread_create(&th[k], NULL, render_thread, &jobs[k]);
        for (int32_t k = 0; k < nthreads; ++k)
            pthread_join(th[k], NULL);
    }
    free(jobs);
    free(th);
    return JLO_OK;
}

/*
 * Rows row0 .. row1-1 of the same W x H frame (single thread); counts holds
 * (row1 - row0) * W values.  Used to check sampled rows of large frames.
 */
int jlo_render_rows(double cr, double ci, double xmin, double xmax, double ymin, double ymax,
                    int32_t W, int32_t H, int32_t max_iter, int32_t mode, int32_t precision,
                    int32_t row0, int32_t row1, uint16_t *counts)
{
    if (W < 1 || H < 1 || max_iter < 1 || max_iter > 65535 || !counts)
        return JLO_EINVAL;
    if (row0 < 0 || row1 > H || row0 >= row1 || (mode != 0 && mode != 1) || (precision != 0 && precision != 1))
        return JLO_EINVAL;
    job_t jb;
    jb.cr = cr; jb.ci = ci;
    jb.xmin = xmin; jb.xmax = xmax; jb.ymin = ymin; jb.ymax = ymax;
    jb.W = W; jb.H = H; jb.max_iter = max_iter; jb.mode = mode; jb.precision = precision;
    jb.row0 = row0; jb.row1 = row1;
    jb.out_row_base = row0;
    jb.counts = counts;
    render_rows(&jb);
    return JLO_OK;
}

typedef struct {
    job_t base;
    int32_t row_start, row_stride, n_rows, first, step;
} strided_t;

/* Thread body: sample rows k = first, first + step, ... < n_rows. */
static void *strided_worker(void *arg)
{
    const strided_t *st = (const strided_t *)arg;
    for (int32_t k = st->first; k < st->n_rows; k += st->step) {
        job_t jb = st->base;
        jb.row0 = st->row_start + k * st->row_stride;
        jb.row1 = jb.row0 + 1;
        jb.out_row_base = jb.row0 - k;  /* sample row k lands at counts[k * W] */
        render_rows(&jb);
    }
    return NULL;
}

/*
 * Rows row_start + k*row_stride, k = 0 .. n_rows-1, of a W x H frame, split
 * over nthreads POSIX threads (rows interleaved); counts holds n_rows * W
 * values.  Used for the bounded CPU timing sample.
 */
int jlo_render_strided(double cr, double ci, double xmin, double xmax, double ymin, double ymax,
                       int32_t W, int32_t H, int32_t max_iter, int32_t mode, int32_t precision,
                       int32_t row_start, int32_t row_stride, int32_t n_rows, uint16_t *counts,
                       int32_t nthreads)
{
    if (W < 1 || H < 1 || max_iter < 1 || max_iter > 65535 || !counts || n_rows < 1 || row_stride < 1)
        return JLO_EINVAL;
    if (row_start < 0 || (int64_t)row_start + (int64_t)(n_rows - 1) * row_stride >= H)
        return JLO_EINVAL;
    if ((mode != 0 && mode != 1) || (precision != 0 && precision != 1))
        return JLO_EINVAL;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > n_rows)
        nthreads = n_rows;
    strided_t *jobs = (strided_t *)calloc((size_t)nthreads, sizeof(strided_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return JLO_EINVAL;
    }
    for (int32_t t = 0; t < nthreads; ++t) {
        job_t *jb = &jobs[t].base;
        jb->cr = cr; jb->ci = ci;
        jb->xmin = xmin; jb->xmax = xmax; jb->ymin = ymin; jb->ymax = ymax;
        jb->W = W; jb->H = H; jb->max_iter = max_iter; jb->mode = mode; jb->precision = precision;
        jb->counts = counts;
        jobs[t].row_start = row_start;
        jobs[t].row_stride = row_stride;
        jobs[t].n_rows = n_rows;
        jobs[t].first = t;
        jobs[t].step = nthreads;
    }
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, strided_worker, &jobs[t]);
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return JLO_OK;
}

/* Escape count of a single point given directly in the working precision
 * (used by tests that choose Z_0 and C themselves). */
int32_t jlo_escape_point(double x, double y, double cr, double ci, int32_t max_iter,
                         int32_t precision)
{
    if (precision == 0)
        return escape_f32((float)x, (float)y, (float)cr, (float)ci, max_iter);
    return escape_f64(x, y, cr, ci, max_iter);
}

/*
 * Colour levels (Sec. 2): count n -> palette entry 255 when n == max_iter
 * (never escaped), else (n * 255) / max_iter in unsigned integer arithmetic.
 * palette: 256 x RGBA8 bytes; rgba: n_pix x 4 bytes out.
 */
int jlo_colour(const uint16_t *counts, int64_t n_pix, int32_t max_iter,
               const uint8_t *palette, uint8_t *rgba)
{
    if (max_iter < 1 || !counts || !palette || !rgba || n_pix < 0)
        return JLO_EINVAL;
    for (int64_t p = 0; p < n_pix; ++p) {
        uint32_t n = counts[p];
        uint32_t idx = (n >= (uint32_t)max_iter) ? 255u : (n * 255u) / (uint32_t)max_iter;
        memcpy(rgba + 4 * p, palette + 4 * idx, 4);
    }
    return JLO_OK;
}

/*
 * Normalised escape-count histogram: hist[b] = #{pixels with count b} / n_pix,
 * the quotient taken in binary64 and rounded once to binary32.
 * hist: max_iter + 1 floats out.
 */
int jlo_hist(const uint16_t *counts, int64_t n_pix, int32_t max_iter, float *hist)
{
    if (max_iter < 1 || !counts || !hist || n_pix < 1)
        return JLO_EINVAL;
    int64_t *bins = (int64_t *)calloc((size_t)max_iter + 1, sizeof(int64_t));
    if (!bins)
        return JLO_EINVAL;
    for (int64_t p = 0; p < n_pix; ++p) {
        uint32_t n = counts[p];
        if (n > (uint32_t)max_iter)
            n = (uint32_t)max_iter;
        bins[n] += 1;
    }
    for (int32_t b = 0; b <= max_iter; ++b)
        hist[b] = (float)((double)bins[b] / (double)n_pix);
    free(bins);
    return JLO_OK;
}
