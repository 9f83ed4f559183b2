// Exact binary64 multiply, square and add on the integer pipes.
//
// The binary64 pipe of this part issues ~1.7 lane operations per clock per
// SM, while 32-bit integer logic/add runs at ~123 and multiply-add at ~64.
// These routines reproduce IEEE 754 binary64 round-to-nearest-even results
// bit for bit for finite normal operands and zeros whose result is zero or a
// normal number; anything else (subnormal or non-finite operands, results
// that underflow below the normal range or overflow) sets `sp` and returns
// an unspecified value -- the caller then redoes the work with the hardware
// instructions.  No FMA is involved anywhere.
//
// Significands are 53-bit integers (implicit bit included); products are
// formed from four (three for squares) 32x32->64 partial products.
#pragma once

#include <stdint.h>

namespace jl {
namespace f64e {

static constexpr unsigned long long kSign = 0x8000000000000000ull;
static constexpr unsigned long long kMant = 0x000fffffffffffffull;
static constexpr unsigned long long kImpl = 0x0010000000000000ull;

__device__ __forceinline__ unsigned long long bits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double from_bits(unsigned long long b) { return __longlong_as_double((long long)b); }

// 106-bit product of two 53-bit significands: returns (hi, lo), P = hi*2^64 + lo.
__device__ __forceinline__ void mul53(unsigned long long a, unsigned long long b, unsigned long long &hi,
                                      unsigned long long &lo)
{
    const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
    const unsigned b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
    const unsigned long long p00 = (unsigned long long)a0 * b0;
    const unsigned long long p01 = (unsigned long long)a0 * b1;
    const unsigned long long p10 = (unsigned long long)a1 * b0;
    const unsigned long long p11 = (unsigned long long)a1 * b1;
    const unsigned long long mid = p01 + p10;  // < 2^54, no overflow
    lo = p00 + (mid << 32);
    hi = p11 + (mid >> 32) + (lo < p00 ? 1ull : 0ull);
}

__device__ __forceinline__ void sqr53(unsigned long long a, unsigned long long &hi, unsigned long long &lo)
{
    const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
    const unsigned long long p00 = (unsigned long long)a0 * a0;
    const unsigned long long p01 = (unsigned long long)a0 * a1;
    const unsigned long long p11 = (unsigned long long)a1 * a1;
    const unsigned long long mid = p01 << 1;  // < 2^54
    lo = p00 + (mid << 32);
    hi = p11 + (mid >> 32) + (lo < p00 ? 1ull : 0ull);
}

// Round the 106-bit product (hi, lo) in [2^104, 2^106) to 53 bits and pack
// with biased exponent e0 (the exponent when the product is below 2^105).
__device__ __forceinline__ unsigned long long round_pack_product(unsigned long long hi, unsigned long long lo, int e0,
                                                                 unsigned long long sign, bool &sp)
{
    const int top = (int)(hi >> 41) & 1;       // product >= 2^105
    const int sh = 52 + top;
    const int e = e0 + top;
    unsigned long long sig = (hi << (64 - sh)) | (lo >> sh);
    const unsigned long long rem = lo << (64 - sh);  // bits below the significand, left-aligned
    const unsigned long long rb = rem >> 63;
    const unsigned long long st = (rem << 1) != 0ull ? 1ull : 0ull;
    sig += rb & (st | (sig & 1ull));
    const unsigned long long r = ((unsigned long long)(long long)(e - 1) << 52) + sig;
    sp |= (e < 1) || (((r >> 52) & 0x7ffull) == 0x7ffull) || (e > 2046);
    return r | sign;
}

// fl(a * b)
__device__ __forceinline__ double mul(double a, double b, bool &sp)
{
    const unsigned long long ua = bits(a), ub = bits(b);
    const unsigned long long sign = (ua ^ ub) & kSign;
    const int ea = (int)((ua >> 52) & 0x7ffull), eb = (int)((ub >> 52) & 0x7ffull);
    const bool za = (ua << 1) == 0ull, zb = (ub << 1) == 0ull;
    sp |= (ea == 0 && !za) || (eb == 0 && !zb) || ea == 0x7ff || eb == 0x7ff;
    unsigned long long hi, lo;
    mul53((ua & kMant) | kImpl, (ub & kMant) | kImpl, hi, lo);
    bool sp2 = false;
    const unsigned long long r = round_pack_product(hi, lo, ea + eb - 1023, sign, sp2);
    const bool zero = za || zb;
    sp |= sp2 && !zero;
    return from_bits(zero ? sign : r);
}

// fl(a * a)
__device__ __forceinline__ double sqr(double a, bool &sp)
{
    const unsigned long long ua = bits(a);
    const int ea = (int)((ua >> 52) & 0x7ffull);
    const bool za = (ua << 1) == 0ull;
    sp |= (ea == 0 && !za) || ea == 0x7ff;
    unsigned long long hi, lo;
    sqr53((ua & kMant) | kImpl, hi, lo);
    bool sp2 = false;
    const unsigned long long r = round_pack_product(hi, lo, 2 * ea - 1023, 0ull, sp2);
    sp |= sp2 && !za;
    return from_bits(za ? 0ull : r);
}

// fl(a + b)
__device__ __forceinline__ double add(double a, double b, bool &sp)
{
    unsigned long long ua = bits(a), ub = bits(b);
    const unsigned long long ma = ua & ~kSign, mb = ub & ~kSign;
    // x: the operand of larger magnitude
    const bool swp = mb > ma;
    const unsigned long long x = swp ? ub : ua;
    const unsigned long long y = swp ? ua : ub;
    const int ex = (int)((x >> 52) & 0x7ffull), ey = (int)((y >> 52) & 0x7ffull);
    const bool zx = (x << 1) == 0ull;   // x == +-0 (then y is zero too)
    const bool zy = (y << 1) == 0ull;   // y == +-0
    sp |= ex == 0x7ff || (ey == 0 && !zy) || (ex == 0 && !zx);
    const unsigned long long sx = x & kSign;
    const bool sub = ((x ^ y) & kSign) != 0ull;
    // significands at bits 62..10 (10 guard bits)
    const unsigned long long MX = zx ? 0ull : (((x & kMant) | kImpl) << 10);
    unsigned long long MY = zy ? 0ull : (((y & kMant) | kImpl) << 10);
    const int d = ex - ey;
    if (d >= 64) {
        MY = MY != 0ull ? 1ull : 0ull;
    } else if (d > 0) {
        const unsigned long long lost = MY << (64 - d);
        MY = (MY >> d) | (lost != 0ull ? 1ull : 0ull);
    }
    const unsigned long long R = sub ? MX - MY : MX + MY;
    // normalise so the leading one sits at bit 62
    const int lz = __clzll((long long)R);   // 64 when R == 0
    unsigned long long N;
    if (lz == 0) {
        N = (R >> 1) | (R & 1ull);          // carry out of an addition
    } else {
        N = R << (lz - 1);                  // exact: cancellation only when no bits were shifted out
    }
    const int e = ex + 1 - lz;
    unsigned long long sig = N >> 10;
    const unsigned long long rb = (N >> 9) & 1ull;
    const unsigned long long st = (N & 0x1ffull) != 0ull ? 1ull : 0ull;
    sig += rb & (st | (sig & 1ull));
    const unsigned long long r = ((unsigned long long)(long long)(e - 1) << 52) + sig;
    const bool zr = R == 0ull;
    if (!zr)
        sp |= (e < 1) || (((r >> 52) & 0x7ffull) == 0x7ffull);
    // exact zero: +0, except (-0) + (-0) = -0
    const unsigned long long zres = ((ua & ub) & kSign);
    return from_bits(zr ? zres : (r | sx));
}

}  // namespace f64e
}  // namespace jl
