// Device helpers shared by the escape-time kernels (jl_escape.cu, jl_map.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jl {

// x + x for binary64 on the integer pipes (the binary64 pipe is narrow on
// this part).  Doubling is exact in IEEE arithmetic, so the bit pattern can be
// formed directly: zero/subnormal -> magnitude shifted left by one (a carry
// into the exponent field gives the correct normal number); exponent field
// 1..2045 -> exponent + 1; 2046 -> signed infinity (what round-to-nearest
// gives on overflow); 2047 (inf, NaN) -> unchanged (NaN stays NaN).  Only
// 32-bit operations on the two words: a 64-bit integer add was measured to
// occupy the binary64 unit (one more binary64-pipe operation per step, the
// same count as a binary64 x + x).
__device__ __forceinline__ double dbl2(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x);
    const uint32_t lo = (uint32_t)__double2loint(x);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7ffu;
    // exponent + 1: 2^52 has a zero low word, so only the high word changes
    uint32_t rhi = hi + (1u << 20), rlo = lo;
    if (e == 0) {
        // magnitude (hi & 0x7fffffff, lo) shifted left by one, below 2^53
        rhi = sign | ((hi & 0x7fffffffu) << 1) | (lo >> 31);
        rlo = lo << 1;
    }
    if (e == 2046) {
        rhi = sign | 0x7ff00000u;
        rlo = 0u;
    }
    if (e == 2047) {
        rhi = hi;
        rlo = lo;
    }
    return __hiloint2double((int)rhi, (int)rlo);
}

// Binary32 estimate of a non-negative binary64 value from its high word,
// truncated (never above the true value, relative error < 2^-20); 0 below
// 2^-126, +inf at or above 2^128.
__device__ __forceinline__ float hi_estimate(double v)
{
    int h = __double2hiint(v) & 0x7fffffff;
    h -= 0x38000000;                 // rebias exponent 1023 -> 127
    h = max(h, 0);
    h = min(h, 0x0ff00000);          // exponent 255 -> +inf
    return __int_as_float(h << 3);
}

// Integer quotient (n * 255) / d for n <= d <= 65535 via a 40-bit reciprocal:
// m = floor(2^40 / d) + 1 gives floor(n*255*m / 2^40) == floor(n*255 / d)
// because the excess n*255*(m - 2^40/d)/2^40 < 2^-16 < 1/d.
__device__ __forceinline__ uint32_t colour_index(uint32_t count, uint32_t max_iter, uint64_t magic)
{
    if (count >= max_iter)
        return 255u;
    uint64_t p = (uint64_t)(count * 255u) * magic;
    return (uint32_t)(p >> 40);
}

}  // namespace jl
