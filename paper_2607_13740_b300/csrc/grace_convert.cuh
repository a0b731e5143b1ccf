// FP64 <-> FP32 conversions on the integer pipe.
//
// On this part the FP64 unit also performs the F2F conversions and runs at
// roughly 1/70 of the FP32 rate, so a kernel that converts every coefficient of
// the FP64 state is bound by the conversions alone.  These routines assemble the
// IEEE-754 bit patterns directly from the sign, exponent and mantissa fields
// (binary64: 1/11/52 bits, bias 1023; binary32: 1/8/23 bits, bias 127) with
// integer operations.
#pragma once

#include <cstdint>

namespace grace {

// binary64 -> binary32, round to nearest even; magnitudes below the binary32
// normal range (2^-126) become a signed zero, above it a signed infinity.
__device__ __forceinline__ float d2f_fast(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
    const uint32_t rest = lo & 0x1FFFFFFFu;                   // the 29 bits dropped
    uint32_t r = ((uint32_t)(e - 896) << 23) | m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    if (e < 897) r = 0u;
    if (e > 1150) r = 0x7F800000u | ((e == 0x7FF && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u);
    return __uint_as_float(sign | r);
}

// binary32 -> binary64, exact, integer operations only (subnormal inputs are
// renormalised with a count of leading zeros).
__device__ __forceinline__ double f2d_fast(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu, sign = u & 0x80000000u;
    // normal (and inf / nan: exponent all ones maps to all ones)
    uint32_t hi = sign | ((e == 0xFFu ? 0x7FFu : e + 896u) << 20) | (m >> 3);
    uint32_t lo = m << 29;
    if (e == 0u) {
        // zero, or subnormal m * 2^-149 = 1.frac * 2^(b - 149) with b the top set bit of m
        const int sh = __clz((int)m) - 8;                   // brings the top bit to bit 23
        const uint32_t fr = (m << sh) & 0x7FFFFFu;
        const uint32_t ed = (uint32_t)(1023 - 126 - sh);    // b - 149 + 1023 with b = 23 - sh
        hi = m ? (sign | (ed << 20) | (fr >> 3)) : sign;
        lo = m ? fr << 29 : 0u;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// true for +-inf and nan (exponent field all ones)
__device__ __forceinline__ bool nonfinite_bits(double d)
{
    return ((uint32_t)((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FFu) == 0x7FFu;
}

__device__ __forceinline__ bool nonfinite_bits(float f) { return (__float_as_uint(f) & 0x7F800000u) == 0x7F800000u; }

// d < 0 (false for -0.0 and nan), by bits
__device__ __forceinline__ bool negative_bits(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned long long mag = u & 0x7FFFFFFFFFFFFFFFull;
    return (u >> 63) && mag != 0ull && mag <= 0x7FF0000000000000ull;
}

// d <= 0 (false for NaN), on the integer pipe: as signed integers the encodings of
// -0 ... -inf lie at or below that of -inf, negative NaNs above it, and +0 is 0
__device__ __forceinline__ bool nonpositive_bits(double d)
{
    const long long b = __double_as_longlong(d);
    return b <= (long long)0xFFF0000000000000ull || b == 0ll;
}

// f * 2^s for a binary32 f (s may be large); results below 2^-126 become 0,
// above the range +-inf.  Zero stays zero.
__device__ __forceinline__ float scale_pow2(float f, int s)
{
    const uint32_t u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFFu);
    if (e == 0) return 0.f;
    const int ne = e + s;
    if (ne <= 0) return 0.f;
    if (ne >= 255) return __uint_as_float((u & 0x80000000u) | 0x7F800000u);
    return __uint_as_float((u & 0x807FFFFFu) | ((uint32_t)ne << 23));
}

// binary64 d * 2^s converted to binary32 (round to nearest even, the same range
// rules as d2f_fast); the exponent shift is exact for results in the binary64
// normal range.
__device__ __forceinline__ float d2f_scaled(double d, int s)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((u >> 52) & 0x7FFull);
    if (e == 0 || e == 0x7FF) return d2f_fast(d);   // zero, subnormal, inf, nan: no shift needed / possible
    const int ne = e + s;
    if (ne <= 0) return __uint_as_float((uint32_t)(u >> 32) & 0x80000000u);
    if (ne >= 0x7FF) return __uint_as_float(((uint32_t)(u >> 32) & 0x80000000u) | 0x7F800000u);
    return d2f_fast(__longlong_as_double((long long)((u & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)ne << 52))));
}

}  // namespace grace
