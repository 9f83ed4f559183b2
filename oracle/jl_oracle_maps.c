/*
 * CPU oracle for generic escape-time maps (TEST INFRASTRUCTURE ONLY; same
 * rules as jl_oracle.c: only tests/, the smoke check and the benchmark's CPU
 * legs may load it, and it shares nothing with the CUDA sources).
 *
 * Sec. 2 uses Z^2 + C and notes that many other functions give fractal
 * images; Fig. 4 shows a rational map and Sec. 5 plans freer functional
 * forms.  Two families:
 *   kind 0, power:    Z <- Z^d + C, integer d in 2..16;
 *   kind 1, rational: Z <- P(Z) / Q(Z) + C, P and Q polynomials with complex
 *                     coefficients of degree 0..8.
 * The count rule is the one of Sec. 2 with the escape radius as a parameter:
 * the number of updates made before the first step whose |Z|^2 is not
 * <= bailout (4 gives the radius 2 of the quadratic map).  Region covering,
 * orientation and rounding of C and the pixel centres are those of
 * jl_oracle.c; in parameter-plane mode Z_0 is the map's z0 (a critical point,
 * 0 for Z^d) and C is the pixel.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#define JLO_OK 0
#define JLO_EINVAL 1

typedef struct {
    int32_t kind;        /* 0 power, 1 rational */
    int32_t degree;      /* power: d */
    int32_t num_degree;  /* rational: degree of P */
    int32_t den_degree;  /* rational: degree of Q */
    double num[18];      /* P: (re, im) pairs, constant term first */
    double den[18];      /* Q: (re, im) pairs, constant term first */
    double bailout;
    double z0r, z0i;
} jlo_map;

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)

#define REAL float
#define SFX f32
#include "map_iter.inc"
#undef REAL
#undef SFX

#define REAL double
#define SFX f64
#include "map_iter.inc"
#undef REAL
#undef SFX

static int map_valid(const jlo_map *m)
{
    if (!m)
        return 0;
    if (m->kind == 0)
        return m->degree >= 2 && m->degree <= 16 && m->bailout > 0.0 && m->bailout < 1e300;
    if (m->kind != 1 || m->num_degree < 0 || m->num_degree > 8 || m->den_degree < 0 || m->den_degree > 8)
        return 0;
    return m->bailout > 0.0 && m->bailout < 1e300;
}

typedef struct {
    const jlo_map *m;
    double cr, ci, xmin, xmax, ymin, ymax;
    int32_t W, H, max_iter, mode, precision, row0, row1;
    uint16_t *counts;
} map_job_t;

static void *map_rows(void *arg)
{
    const map_job_t *jb = (const map_job_t *)arg;
    const double dx = (jb->xmax - jb->xmin) / (double)jb->W;
    const double dy = (jb->ymax - jb->ymin) / (double)jb->H;
    for (int32_t j = jb->row0; j < jb->row1; ++j) {
        double yd = jb->ymin + ((double)j + 0.5) * dy;
        for (int32_t i = 0; i < jb->W; ++i) {
            double xd = jb->xmin + ((double)i + 0.5) * dx;
            int32_t n;
            if (jb->precision == 0) {
                if (jb->mode == 0)
                    n = map_escape_f32(jb->m, (float)xd, (float)yd, (float)jb->cr, (float)jb->ci, jb->max_iter);
                else
                    n = map_escape_f32(jb->m, (float)jb->m->z0r, (float)jb->m->z0i, (float)xd, (float)yd,
                                       jb->max_iter);
            } else {
                if (jb->mode == 0)
                    n = map_escape_f64(jb->m, xd, yd, jb->cr, jb->ci, jb->max_iter);
                else
                    n = map_escape_f64(jb->m, jb->m->z0r, jb->m->z0i, xd, yd, jb->max_iter);
            }
            jb->counts[(size_t)j * (size_t)jb->W + (size_t)i] = (uint16_t)n;
        }
    }
    return NULL;
}

/*
 * Escape counts of a W x H grid under the map m (uint16, row-major, row 0 at
 * y = ymin); mode 0: Z_0 = pixel, C = (cr, ci); mode 1: Z_0 = (z0r, z0i),
 * C = pixel.  precision 0 = binary32, 1 = binary64.  Rows are split into
 * contiguous bands over nthreads POSIX threads.  Returns 0 or 1 (invalid).
 */
int jlo_render_map(const jlo_map *m, double cr, double ci, double xmin, double xmax, double ymin, double ymax,
                   int32_t W, int32_t H, int32_t max_iter, int32_t mode, int32_t precision, uint16_t *counts,
                   int32_t nthreads)
{
    if (!map_valid(m) || W < 1 || H < 1 || max_iter < 1 || max_iter > 65535 || !counts)
        return JLO_EINVAL;
    if ((mode != 0 && mode != 1) || (precision != 0 && precision != 1))
        return JLO_EINVAL;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > H)
        nthreads = H;
    map_job_t *jobs = (map_job_t *)calloc((size_t)nthreads, sizeof(map_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return JLO_EINVAL;
    }
    for (int32_t t = 0; t < nthreads; ++t) {
        map_job_t *jb = &jobs[t];
        jb->m = m;
        jb->cr = cr;
        jb->ci = ci;
        jb->xmin = xmin;
        jb->xmax = xmax;
        jb->ymin = ymin;
        jb->ymax = ymax;
        jb->W = W;
        jb->H = H;
        jb->max_iter = max_iter;
        jb->mode = mode;
        jb->precision = precision;
        jb->row0 = (int32_t)((int64_t)H * t / nthreads);
        jb->row1 = (int32_t)((int64_t)H * (t + 1) / nthreads);
        jb->counts = counts;
    }
    for (int32_t t = 1; t < nthreads; ++t)
        pthread_create(&th[t], NULL, map_rows, &jobs[t]);
    map_rows(&jobs[0]);
    for (int32_t t = 1; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return JLO_OK;
}

/* Escape count of one point: Z_0 = (x, y), C = (cr, ci), each rounded once to
 * the working precision.  Returns -1 on invalid arguments. */
int32_t jlo_map_escape_point(const jlo_map *m, double x, double y, double cr, double ci, int32_t max_iter,
                             int32_t precision)
{
    if (!map_valid(m) || max_iter < 1 || max_iter > 65535)
        return -1;
    if (precision == 0)
        return map_escape_f32(m, (float)x, (float)y, (float)cr, (float)ci, max_iter);
    return map_escape_f64(m, x, y, cr, ci, max_iter);
}

/* One update F(Z) + C without the escape test (for checking F itself).
 * out[0], out[1]: the real and imaginary parts, widened to binary64. */
int jlo_map_step(const jlo_map *m, double x, double y, double cr, double ci, int32_t precision, double *out)
{
    if (!map_valid(m) || !out)
        return JLO_EINVAL;
    if (precision == 0) {
        float num[18], den[18], fx, fy;
        round_coeffs_f32(m, num, den);
        map_f_f32(m, num, den, (float)x, (float)y, &fx, &fy);
        out[0] = (double)(fx + (float)cr);
        out[1] = (double)(fy + (float)ci);
    } else {
        double num[18], den[18], fx, fy;
        round_coeffs_f64(m, num, den);
        map_f_f64(m, num, den, x, y, &fx, &fy);
        out[0] = fx + cr;
        out[1] = fy + ci;
    }
    return JLO_OK;
}
