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

}  // namespace jl

using namespace jl;

extern "C" int jl_probe_peak(int32_t precision, int32_t iters, double *lane_ops_per_s, double *seconds,
                             void *stream)
{
    if (precision != JL_FP32 && precision != JL_FP64)
        return fail(JL_EINVAL, "precision must be JL_FP32 or JL_FP64");
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
        if (precision == JL_FP32)
            fp_probe_kernel<float><<<grid, threads, 0, st>>>((float *)out, iters, 0.999f, 0.001f);
        else
            fp_probe_kernel<double><<<grid, threads, 0, st>>>((double *)out, iters, 0.999, 0.001);
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
        const double ops = (double)grid * threads * (double)iters * 8.0 * 2.0;
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
