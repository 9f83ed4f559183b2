// Issue-rate probe for the binary32 and binary64 pipes: the denominators of
// the escape kernels' ALU roofline.  Each thread runs 8 independent chains of
// v = v*a + b written as a separate multiply and add (no FMA), so every lane
// operation is one FMUL/FADD (DMUL/DADD) and the chains hide the latency.
#include <cuda_runtime.h>
#include <stdint.h>

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

// Packed binary32 pairs (add/mul.rn.f32x2, sm_100 and later), kind 2:
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

}  // namespace jl

using namespace jl;

extern "C" int jl_probe_peak(int32_t kind, int32_t iters, double *lane_ops_per_s, double *seconds, void *stream)
{
    if (kind < 0 || kind > 2)
        return fail(JL_EINVAL, "kind must be 0 (binary32), 1 (binary64) or 2 (packed binary32 pairs)");
    if (iters < 1 || !lane_ops_per_s)
        return fail(JL_EINVAL, "iters must be >= 1 and lane_ops_per_s non-NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = device_sm_count();
    if (sms <= 0)
        return fail(JL_EUNSUPPORTED, "no CUDA device");
    const int threads = 256;
    const int grid = sms * 8;
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
        if (kind == 0)
            fp_probe_kernel<float><<<grid, threads, 0, st>>>((float *)out, iters, 0.999f, 0.001f);
        else if (kind == 1)
            fp_probe_kernel<double><<<grid, threads, 0, st>>>((double *)out, iters, 0.999, 0.001);
        else
            f32x2_probe_kernel<<<grid, threads, 0, st>>>((unsigned long long *)out, iters, 0.999f, 0.001f);
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
        // 8 chains per thread, two lane operations per chain step (a multiply
        // and an add; for kind 2 one packed instruction of two lanes)
        const double ops = (double)grid * threads * (double)iters * 16.0;
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
