// Issue-rate probe for the binary32 and binary64 pipes: the denominators of
// the escape kernels' ALU roofline.  Each thread runs 8 independent chains of
// v = v*a + b written as a separate multiply and add (no FMA), so every lane
// operation is one FMUL/FADD (DMUL/DADD) and the chains hide the latency.
#include <cuda_runtime.h>
#include <stdint.h>

#include "jl_common.cuh"
#include "jl_internal.h"

namespace jl {

template <typename T>
__global__ void __launch_bounds__(256) fp_probe_kernel(T *out, int iters, T a, T b)
{
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (sizeof(T) == 4)
                v[k] = __fadd_rn(__fmul_rn(v[k], a), b);
            else
                v[k] = __dadd_rn(__dmul_rn(v[k], a), b);
        }
    }
    T s = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k)
        s = s + v[k];
    if (s == (T)12345.678)  // practically never; keeps the chains live
        out[blockIdx.x] = s;
}

// Integer pipe probes: kind 2 = xor + add (logic/add pipe), kind 3 = 32-bit
// multiply-add, kind 4 = high half of a 32x32 product.  One lane op per
// statement; 8 independent chains per thread.
template <int KIND>
__global__ void __launch_bounds__(256) int_probe_kernel(uint32_t *out, int iters, uint32_t a, uint32_t b)
{
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = threadIdx.x * 2654435761u + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (KIND == 2) {
                v[k] = (v[k] ^ a) + b;
                asm volatile("" : "+r"(v[k]));
            } else if constexpr (KIND == 3) {
                v[k] = v[k] * a + b;
            } else {
                v[k] = __umulhi(v[k], a) ^ b;
            }
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        s ^= v[k];
    if (s == 0x9e3779b9u)
        out[blockIdx.x] = s;
}

// Packed binary32 pairs (add/mul.rn.f32x2, sm_100 and later), kind 5:
// four chains of packed adds and four of packed multiplies per thread, so
// no product ever feeds a sum (the compiler contracts a packed multiply and
// a following packed add into one fused operation).  Each instruction is two
// binary32 lane operations; the probe tells whether packing raises the
// lane-operation rate of separately rounded adds and multiplies.  (Measured
// on this part: it does not; a packed instruction holds the pipe twice as
// long as a scalar one.)
__device__ __forceinline__ unsigned long long mul_f32x2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__global__ void __launch_bounds__(256) f32x2_probe_kernel(unsigned long long *out, int iters, float a, float b)
{
    const unsigned long long a2 = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
    const unsigned long long b2 = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
    unsigned long long v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float lo = (float)(threadIdx.x + k) * 1e-3f, hi = (float)(threadIdx.x + 2 * k) * 1e-3f;
        v[k] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = (k & 1) ? mul_f32x2(v[k], a2) : add_f32x2(v[k], b2);
    }
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        s ^= v[k];
    if (s == 0x9e3779b97f4a7c15ull)
        out[blockIdx.x] = s;
}

// 64-bit integer probes: kind 6 = 64-bit add chains, kind 7 = 64-bit
// shift-and-xor chains, kind 8 = 64-bit compare-and-select chains.  They tell
// which pipe the 64-bit integer forms use (the integer-pipe binary64
// arithmetic is built from them).
template <int KIND>
__global__ void __launch_bounds__(256) int64_probe_kernel(unsigned long long *out, int iters, unsigned long long a,
                                                          unsigned long long b)
{
    unsigned long long v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = (unsigned long long)threadIdx.x * 0x9e3779b97f4a7c15ull + k;
    const int s = (int)(a & 31ull) + 1;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (KIND == 6) {
                v[k] = v[k] + a;
                asm volatile("" : "+l"(v[k]));
            } else if constexpr (KIND == 7) {
                v[k] = (v[k] << s) ^ (v[k] >> (s + 3));
            } else {
                v[k] = (v[k] > a) ? v[k] - b : v[k] + a;
            }
        }
    }
    unsigned long long t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        t ^= v[k];
    if (t == 0x9e3779b97f4a7c15ull)
        out[blockIdx.x] = t;
}

// binary64 fused multiply-add chains, kind 9: v = fma(v, a, b), one DFMA per
// chain step (the lane-refill kernel's steps have exact fused forms; this
// tells the rate of that instruction against kind 1's separate DMUL + DADD).
__global__ void __launch_bounds__(256) dfma_probe_kernel(double *out, int iters, double a, double b)
{
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = __fma_rn(v[k], a, b);
    }
    double s = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k)
        s = s + v[k];
    if (s == 12345.678)
        out[blockIdx.x] = s;
}

// binary64 escape steps, kinds 10 and 11: two independent chains per thread
// (as the lane-refill kernel's two pixel slots) of Z <- Z^2 + C formed as
// that kernel forms them: products x*x, y*y and (2x)*y, sums (x2 - y2) + cr
// and t + ci, 2x on the integer pipe (dbl2); six binary64 lane operations per
// step.  Kind 11 adds the kernel's per-step binary32 estimate of |Z|^2 and its
// counters.  No refill, service or stores: the step's own ceiling.  C in the
// main cardioid keeps every orbit bounded (and away from subnormals).
template <bool TEST>
__global__ void __launch_bounds__(256) escape_step_probe_kernel(double *out, int iters, double cr, double ci)
{
    double x[2], y[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        x[k] = (double)(threadIdx.x + 7 * k) * 1e-4;
        y[k] = (double)(blockIdx.x & 255) * 1e-4 + k * 1e-3;
    }
    int cnt = 0;
    bool amb = false;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const double x2 = __dmul_rn(x[k], x[k]);
            const double y2 = __dmul_rn(y[k], y[k]);
            if constexpr (TEST) {
                const float r32 = __fadd_rn(hi_estimate(x2), hi_estimate(y2));
                cnt += (r32 < 3.9999847412109375f) ? 1 : 0;
                amb |= (r32 >= 3.9999847412109375f) & (r32 <= 4.0000152587890625f);
            }
            const double t = __dmul_rn(dbl2(x[k]), y[k]);
            y[k] = __dadd_rn(t, ci);
            x[k] = __dadd_rn(__dsub_rn(x2, y2), cr);
        }
    }
    const double s = __dadd_rn(__dadd_rn(x[0], x[1]), __dadd_rn(y[0], y[1]));
    if (s == 12345.678 || cnt == 7 || amb)  // practically never; keeps the chains live
        out[blockIdx.x] = s + cnt;
}

}  // namespace jl

using namespace jl;

extern "C" int jl_probe_peak(int32_t precision, int32_t iters, double *lane_ops_per_s, double *seconds,
                             void *stream)
{
    if (precision < 0 || precision > 13)
        return fail(JL_EINVAL, "kind must be 0 (binary32), 1 (binary64), 2 (int xor+add), 3 (int mad), 4 (int mulhi), "
                               "5 (packed binary32 pairs), 6 (int64 add), 7 (int64 shift+xor), 8 (int64 compare+select), "
                               "9 (binary64 fused multiply-add), 10 (binary64 escape step), "
                               "11 (binary64 escape step with the binary32 test), 12 / 13 (kind 10 with 4 / 6 "
                               "warps per scheduler)");
    if (iters < 1 || !lane_ops_per_s)
        return fail(JL_EINVAL, "iters must be >= 1 and lane_ops_per_s non-NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = device_sm_count();
    if (sms <= 0)
        return fail(JL_EUNSUPPORTED, "no CUDA device");
    const int threads = 256;
    // kinds 12 and 13: two or three CTAs of 256 threads per SM, i.e. 4 or 6
    // warps per scheduler (the lane-refill kernel runs about 4)
    const int grid = sms * (precision == 12 ? 2 : precision == 13 ? 3 : 8);
    void *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, (size_t)grid * 8, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(probe)");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    int rc = JL_OK;
    for (int rep = 0; rep < 2 && rc == JL_OK; ++rep) {  // first launch warms up
        cudaEventRecord(t0, st);
        if (precision == JL_FP32)
            fp_probe_kernel<float><<<grid, threads, 0, st>>>((float *)out, iters, 0.999f, 0.001f);
        else if (precision == JL_FP64)
            fp_probe_kernel<double><<<grid, threads, 0, st>>>((double *)out, iters, 0.999, 0.001);
        else if (precision == 2)
            int_probe_kernel<2><<<grid, threads, 0, st>>>((uint32_t *)out, iters, 0x5bd1e995u, 0x1b873593u);
        else if (precision == 3)
            int_probe_kernel<3><<<grid, threads, 0, st>>>((uint32_t *)out, iters, 0x5bd1e995u, 0x1b873593u);
        else if (precision == 5)
            f32x2_probe_kernel<<<grid, threads, 0, st>>>((unsigned long long *)out, iters, 0.999f, 0.001f);
        else if (precision == 6)
            int64_probe_kernel<6><<<grid, threads, 0, st>>>((unsigned long long *)out, iters, 0x9e3779b97f4a7c15ull, 7ull);
        else if (precision == 7)
            int64_probe_kernel<7><<<grid, threads, 0, st>>>((unsigned long long *)out, iters, 0x5ull, 7ull);
        else if (precision == 8)
            int64_probe_kernel<8><<<grid, threads, 0, st>>>((unsigned long long *)out, iters, 0x7fffffffffffull, 0x12345ull);
        else if (precision == 9)
            dfma_probe_kernel<<<grid, threads, 0, st>>>((double *)out, iters, 0.999, 0.001);
        else if (precision == 10 || precision == 12 || precision == 13)
            escape_step_probe_kernel<false><<<grid, threads, 0, st>>>((double *)out, iters, -0.1, 0.1);
        else if (precision == 11)
            escape_step_probe_kernel<true><<<grid, threads, 0, st>>>((double *)out, iters, -0.1, 0.1);
        else
            int_probe_kernel<4><<<grid, threads, 0, st>>>((uint32_t *)out, iters, 0x5bd1e995u, 0x1b873593u);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            rc = cuda_fail(e, "probe launch");
        cudaEventRecord(t1, st);
    }
    if (rc == JL_OK) {
        e = cudaEventSynchronize(t1);
        if (e != cudaSuccess)
            rc = cuda_fail(e, "probe sync");
    }
    if (rc == JL_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        // lane ops per chain step (64-bit kinds: one 64-bit operation per step
        // for add, two shifts and an xor, a compare and a select plus the add)
        // (escape steps: two chains of six binary64 operations per step)
        const double per =
            (precision == 3 || precision == 6 || precision == 9) ? 1.0 : (precision == 7 ? 3.0 : 2.0);
        const double chains_x_per = precision >= 10 ? 2.0 * 6.0 : 8.0 * per;
        const double ops = (double)grid * threads * (double)iters * chains_x_per;
        *lane_ops_per_s = ops / (ms * 1e-3);
        if (seconds)
            *seconds = ms * 1e-3;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    return rc;
}
