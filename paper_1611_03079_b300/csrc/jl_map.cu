// Generic escape-time maps (paper Sec. 2: other functions than Z^2 + C;
// Fig. 4: a rational map; Sec. 5: freer functional forms).
//
//   power     Z <- Z^d + C, 2 <= d <= 16
//   rational  Z <- P(Z) / Q(Z) + C, deg P, deg Q <= 8, complex coefficients
//
// One step in the working type T (every operation an explicit
// round-to-nearest intrinsic, never contracted):
//   x2 = x*x; y2 = y*y; escape unless x2 + y2 <= bailout;
//   (fx, fy) = F(x, y); x = fx + cr; y = fy + ci.
// F for the power map is square-and-multiply over the bits of d from the
// leading one down; the first square reuses x2 and y2, which are the same
// rounded products the square would form.  F for the rational map is Horner
// for P and Q followed by the quotient (P conj Q) / |Q|^2 with correctly
// rounded division.
//
// Kernel shape: the static tile kernel of the quadratic path (persistent
// CTAs over 32 x 32 pixel tiles, four pixels per thread, exact test at every
// step and per-lane exit) with the map's step in place of Z^2 + C.  Degrees
// 2..8 of the power map are compile-time (unrolled square-and-multiply);
// larger degrees loop over the bits at run time.  Coefficients travel in the
// launch parameters (constant bank), rounded once to T on the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string.h>

#include "jl_common.cuh"
#include "jl_internal.h"

namespace jl {

struct MapArgs {
    Frame F;
    int32_t degree;       // power: d
    int32_t nd, nq;       // rational: degrees of P and Q
    int32_t hist_smem;    // 1: histogram bins in shared memory
    int64_t total_tiles;
    double num64[18], den64[18];
    float num32[18], den32[18];
    double bail64, z0r64, z0i64;
    float bail32, z0r32, z0i32;
    uint32_t palette[256];
};

template <typename T>
struct Arith;
template <>
struct Arith<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float twice(float a) { return __fadd_rn(a, a); }
    static __device__ __forceinline__ const float *num(const MapArgs &m) { return m.num32; }
    static __device__ __forceinline__ const float *den(const MapArgs &m) { return m.den32; }
    static __device__ __forceinline__ float bail(const MapArgs &m) { return m.bail32; }
    static __device__ __forceinline__ float z0r(const MapArgs &m) { return m.z0r32; }
    static __device__ __forceinline__ float z0i(const MapArgs &m) { return m.z0i32; }
    static __device__ __forceinline__ float cr(const Frame &f) { return f.cr32; }
    static __device__ __forceinline__ float ci(const Frame &f) { return f.ci32; }
};
template <>
struct Arith<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double twice(double a) { return dbl2(a); }  // exact, integer pipes
    static __device__ __forceinline__ const double *num(const MapArgs &m) { return m.num64; }
    static __device__ __forceinline__ const double *den(const MapArgs &m) { return m.den64; }
    static __device__ __forceinline__ double bail(const MapArgs &m) { return m.bail64; }
    static __device__ __forceinline__ double z0r(const MapArgs &m) { return m.z0r64; }
    static __device__ __forceinline__ double z0i(const MapArgs &m) { return m.z0i64; }
    static __device__ __forceinline__ double cr(const Frame &f) { return f.cr; }
    static __device__ __forceinline__ double ci(const Frame &f) { return f.ci; }
};

// W <- W * Z: (a c - b d) + (a d + b c) i
template <typename T>
__device__ __forceinline__ void cmul_z(T &wx, T &wy, T x, T y)
{
    using A = Arith<T>;
    const T ac = A::mul(wx, x), bd = A::mul(wy, y), ad = A::mul(wx, y), bc = A::mul(wy, x);
    wx = A::sub(ac, bd);
    wy = A::add(ad, bc);
}

// W <- W^2: (a a - b b) + ((a + a) b) i
template <typename T>
__device__ __forceinline__ void csqr(T &wx, T &wy)
{
    using A = Arith<T>;
    const T a2 = A::mul(wx, wx), b2 = A::mul(wy, wy), t = A::mul(A::twice(wx), wy);
    wx = A::sub(a2, b2);
    wy = t;
}

// Z^d with D = d known at compile time (D >= 2), or D == 0 for a run-time d.
template <typename T, int D>
__device__ __forceinline__ void power_f(T x, T y, T x2, T y2, int d_rt, T &ox, T &oy)
{
    using A = Arith<T>;
    const int d = D ? D : d_rt;
    const int top = 31 - __clz(d);
    // first square from the test's products
    T wx = A::sub(x2, y2), wy = A::mul(A::twice(x), y);
    if ((d >> (top - 1)) & 1)
        cmul_z(wx, wy, x, y);
    if constexpr (D != 0) {
#pragma unroll
        for (int b = top - 2; b >= 0; --b) {
            csqr(wx, wy);
            if ((D >> b) & 1)
                cmul_z(wx, wy, x, y);
        }
    } else {
#pragma unroll 1
        for (int b = top - 2; b >= 0; --b) {
            csqr(wx, wy);
            if ((d >> b) & 1)
                cmul_z(wx, wy, x, y);
        }
    }
    ox = wx;
    oy = wy;
}

// Horner's rule for sum_k a_k Z^k, degree n <= 8, a: (re, im) pairs.
template <typename T>
__device__ __forceinline__ void horner(const T *a, int n, T x, T y, T &pr, T &pi)
{
    using A = Arith<T>;
    pr = a[2 * n];
    pi = a[2 * n + 1];
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        if (k < n) {
            cmul_z(pr, pi, x, y);
            pr = A::add(pr, a[2 * k]);
            pi = A::add(pi, a[2 * k + 1]);
        }
    }
}

template <typename T>
__device__ __forceinline__ void rational_f(const MapArgs &m, T x, T y, T &ox, T &oy)
{
    using A = Arith<T>;
    T pr, pi, qr, qi;
    horner(A::num(m), m.nd, x, y, pr, pi);
    horner(A::den(m), m.nq, x, y, qr, qi);
    const T q2 = A::add(A::mul(qr, qr), A::mul(qi, qi));
    const T nr = A::add(A::mul(pr, qr), A::mul(pi, qi));
    const T ni = A::sub(A::mul(pi, qr), A::mul(pr, qi));
    ox = A::div(nr, q2);
    oy = A::div(ni, q2);
}

// Escape count from Z_0 = (x, y) with constant (cr, ci).  D: -1 rational,
// 0 power with run-time degree, 2..8 power with that degree.
template <typename T, int D>
__device__ __forceinline__ int map_escape(const MapArgs &m, T x, T y, T cr, T ci, int max_iter, T bail)
{
    using A = Arith<T>;
    for (int n = 0; n < max_iter; ++n) {
        const T x2 = A::mul(x, x), y2 = A::mul(y, y);
        const T r = A::add(x2, y2);
        if (!(r <= bail))
            return n;
        T fx, fy;
        if constexpr (D < 0)
            rational_f(m, x, y, fx, fy);
        else
            power_f<T, D>(x, y, x2, y2, m.degree, fx, fy);
        x = A::add(fx, cr);
        y = A::add(fy, ci);
    }
    return max_iter;
}

template <typename T, int D>
__global__ void __launch_bounds__(256) map_kernel(const __grid_constant__ MapArgs a)
{
    using A = Arith<T>;
    __shared__ uint32_t pal[256];
    extern __shared__ uint32_t hbins[];
    const Frame &F = a.F;
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        pal[t] = a.palette[t];
    const int nb = a.hist_smem ? F.max_iter + 1 : 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hbins[t] = 0;
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dxp = (w & 3) * 8 + (lane & 7);
    const int dyp = (w >> 2) * 4 + (lane >> 3);
    const int W = F.W, H = F.H, mi = F.max_iter;
    const bool julia = F.mode == JL_JULIA;
    const T fcr = A::cr(F), fci = A::ci(F), bail = A::bail(a), z0r = A::z0r(a), z0i = A::z0i(a);
    const T *xs = static_cast<const T *>(F.xs);
    const T *ys = static_cast<const T *>(F.ys);
    const bool u8 = F.count_type == JL_COUNT_U8;

    for (long long tile = blockIdx.x; tile < a.total_tiles; tile += gridDim.x) {
        const uint32_t lt = (uint32_t)tile;
        const uint32_t ty = (uint32_t)(((uint64_t)lt * F.tiles_x_magic) >> 40);
        const uint32_t tx = lt - ty * (uint32_t)F.tiles_x;
        const int i = (int)tx * 32 + dxp;
        if (i >= W)
            continue;
        const T xv = xs[i];
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int j = (int)ty * 32 + dyp + 8 * q;
            if (j >= H)
                break;
            const T yv = ys[j];
            const int count = julia ? map_escape<T, D>(a, xv, yv, fcr, fci, mi, bail)
                                    : map_escape<T, D>(a, z0r, z0i, xv, yv, mi, bail);
            const int p = j * W + i;
            if (F.counts) {
                if (u8)
                    F.counts[p] = (uint8_t)count;
                else
                    reinterpret_cast<uint16_t *>(F.counts)[p] = (uint16_t)count;
            }
            if (F.rgba)
                F.rgba[p] = pal[colour_index((uint32_t)count, (uint32_t)mi, F.colour_magic)];
            if (F.hist_bins) {
                if (a.hist_smem) {
                    atomicAdd(&hbins[count], 1u);
                } else {
                    const unsigned act = __activemask();
                    const unsigned grp = __match_any_sync(act, (unsigned)count);
                    if ((grp & ((1u << lane) - 1u)) == 0)
                        atomicAdd(&F.hist_bins[count], (unsigned)__popc(grp));
                }
            }
        }
    }
    if (nb) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const uint32_t v = hbins[t];
            if (v)
                atomicAdd(&F.hist_bins[t], v);
        }
    }
}

template <typename T, int D>
static cudaError_t launch_map_t(const MapArgs &a, cudaStream_t st)
{
    const size_t smem = a.hist_smem ? (size_t)(a.F.max_iter + 1) * sizeof(uint32_t) : 0;
    auto kern = map_kernel<T, D>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    cudaError_t e = occupancy_per_sm(reinterpret_cast<const void *>(kern), 256, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    const int sms = device_sm_count();
    long long grid = (long long)(sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
    if (grid > a.total_tiles)
        grid = a.total_tiles;
    kern<<<(unsigned)grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_map_prec(const MapArgs &a, int kind, cudaStream_t st)
{
    if (kind == JL_MAP_RATIONAL)
        return launch_map_t<T, -1>(a, st);
    switch (a.degree) {
    case 2: return launch_map_t<T, 2>(a, st);
    case 3: return launch_map_t<T, 3>(a, st);
    case 4: return launch_map_t<T, 4>(a, st);
    case 5: return launch_map_t<T, 5>(a, st);
    case 6: return launch_map_t<T, 6>(a, st);
    case 7: return launch_map_t<T, 7>(a, st);
    case 8: return launch_map_t<T, 8>(a, st);
    default: return launch_map_t<T, 0>(a, st);
    }
}

static int validate_map(const jl_map *m)
{
    if (!m)
        return fail(JL_EINVAL, "map must not be NULL");
    if (m->kind == JL_MAP_POWER) {
        if (m->degree < 2 || m->degree > 16)
            return fail(JL_EINVAL, "power map degree must be 2..16");
    } else if (m->kind == JL_MAP_RATIONAL) {
        if (m->num_degree < 0 || m->num_degree > 8 || m->den_degree < 0 || m->den_degree > 8)
            return fail(JL_EINVAL, "rational map degrees must be 0..8");
        for (int k = 0; k < 2 * (m->num_degree + 1); ++k)
            if (!std::isfinite(m->num[k]))
                return fail(JL_EINVAL, "rational map numerator coefficient is not finite");
        for (int k = 0; k < 2 * (m->den_degree + 1); ++k)
            if (!std::isfinite(m->den[k]))
                return fail(JL_EINVAL, "rational map denominator coefficient is not finite");
    } else {
        return fail(JL_EINVAL, "unknown map kind");
    }
    if (!std::isfinite(m->bailout) || !(m->bailout > 0.0))
        return fail(JL_EINVAL, "bailout must be finite and > 0");
    if (!std::isfinite(m->z0r) || !std::isfinite(m->z0i))
        return fail(JL_EINVAL, "z0 must be finite");
    return JL_OK;
}

}  // namespace jl

using namespace jl;

extern "C" int jl_render_map(const jl_map *map, double cr, double ci, jl_rect rect, int32_t width, int32_t height,
                             int32_t max_iter, int32_t precision, int32_t mode, int32_t count_type, void *counts,
                             uint8_t *rgba, const uint8_t *palette, float *hist, void *stream)
{
    int rc = validate_map(map);
    if (rc != JL_OK)
        return rc;
    Frame F;
    int prec = 0;
    rc = make_frame(cr, ci, rect, width, height, max_iter, precision, mode, count_type, counts != nullptr,
                    rgba != nullptr, hist != nullptr, &F, &prec);
    if (rc != JL_OK)
        return rc;
    F.counts = static_cast<uint8_t *>(counts);
    F.rgba = reinterpret_cast<uint32_t *>(rgba);
    F.hist_bins = reinterpret_cast<uint32_t *>(hist);
    const int sms = device_sm_count();
    if (sms <= 0)
        return fail(JL_EUNSUPPORTED, "no CUDA device");

    MapArgs a;
    memset(&a, 0, sizeof(a));
    a.degree = map->kind == JL_MAP_POWER ? map->degree : 0;
    a.nd = map->kind == JL_MAP_RATIONAL ? map->num_degree : 0;
    a.nq = map->kind == JL_MAP_RATIONAL ? map->den_degree : 0;
    for (int k = 0; k < 18; ++k) {
        const double nv = map->kind == JL_MAP_RATIONAL ? map->num[k] : 0.0;
        const double dv = map->kind == JL_MAP_RATIONAL ? map->den[k] : 0.0;
        a.num64[k] = nv;
        a.den64[k] = dv;
        a.num32[k] = (float)nv;  // rounded once, to nearest
        a.den32[k] = (float)dv;
    }
    a.bail64 = map->bailout;
    a.bail32 = (float)map->bailout;
    a.z0r64 = map->z0r;
    a.z0i64 = map->z0i;
    a.z0r32 = (float)map->z0r;
    a.z0i32 = (float)map->z0i;
    a.hist_smem = (F.hist_bins && F.max_iter + 1 <= 4096) ? 1 : 0;
    a.total_tiles = F.tile_count;
    uint8_t pal[1024];
    if (palette)
        memcpy(pal, palette, 1024);
    else
        default_palette_bytes(pal);
    memcpy(a.palette, pal, 1024);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t esz = prec == JL_FP64 ? 8 : 4;
    const size_t coord_bytes = ((size_t)F.W + (size_t)F.H) * esz;
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, coord_bytes, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(coordinate tables)");
    uint8_t *base = static_cast<uint8_t *>(scratch);
    F.xs = base;
    F.ys = base + (size_t)F.W * esz;
    do {
        if (F.hist_bins) {
            e = cudaMemsetAsync(F.hist_bins, 0, ((size_t)F.max_iter + 1) * 4, st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync(hist)"); break; }
        }
        e = launch_coords(nullptr, &F, 1, st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "coords kernel launch"); break; }
        a.F = F;
        e = prec == JL_FP64 ? launch_map_prec<double>(a, map->kind, st) : launch_map_prec<float>(a, map->kind, st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "map kernel launch"); break; }
        if (F.hist_bins) {
            e = launch_hist_finalize(nullptr, &F, 1, st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "histogram finalize launch"); break; }
        }
    } while (0);
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (rc == JL_OK && e2 != cudaSuccess)
        rc = cuda_fail(e2, "cudaFreeAsync(coordinate tables)");
    return rc;
}
