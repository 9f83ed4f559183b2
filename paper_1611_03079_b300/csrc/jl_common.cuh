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
// gives on overflow); 2047 (inf, NaN) -> unchanged (NaN stays NaN).
__device__ __forceinline__ double dbl2(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = b & 0x8000000000000000ull;
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned e = (unsigned)(mag >> 52);
    unsigned long long r = b + (1ull << 52);
    r = (e == 0) ? (sign | (mag << 1)) : r;
    r = (e == 2046) ? (sign | 0x7ff0000000000000ull) : r;
    r = (e == 2047) ? b : r;
    return __longlong_as_double((long long)r);
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
