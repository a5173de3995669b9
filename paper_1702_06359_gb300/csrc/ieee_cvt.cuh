// Conversions between IEEE 754 binary32 and binary64 done with integer operations on the bit
// fields (binary32: sign, 8-bit exponent biased by 127, 23-bit fraction; binary64: sign, 11-bit
// exponent biased by 1023, 52-bit fraction).
//
// The mixed-precision Kalman update moves the 21 covariance terms, the hit geometry and the gain
// between float and double at every update.  This GPU has few double-precision units, and a
// conversion there costs about as much as a double multiply-add, so the update converts with
// integer operations instead.  Float -> double is exact; double -> float rounds to nearest, ties
// to even.  Subnormal inputs and results are flushed to a signed zero, as the single-precision
// arithmetic of this library does (it is compiled to flush them); infinities and NaNs keep their
// class.  Host and device share the code (tests compare it with the C conversions on the host).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace tkf {

__host__ __device__ __forceinline__ uint32_t f32_bits(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float f32_from(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t f64_bits(double d)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double f64_from(uint32_t hi, uint32_t lo)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t u = ((uint64_t)hi << 32) | lo;
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

// binary32 -> binary64 (exact for normal numbers)
__host__ __device__ __forceinline__ double f32_to_f64_bits(float f)
{
    const uint32_t u = f32_bits(f);
    const uint32_t sgn = u & 0x80000000u, a = u & 0x7FFFFFFFu;
    // the exponent rebiased by 1023 - 127 = 896 (0x38000000 in the high word once the fraction
    // has moved 3 bits down); the fraction's 23 bits become the top 23 of the 52
    uint32_t hi = sgn | ((a >> 3) + 0x38000000u), lo = a << 29;
    if (a >= 0x7F800000u) hi = sgn | 0x7FF00000u | ((a & 0x007FFFFFu) >> 3);  // inf, NaN
    if (a < 0x00800000u) {                                                    // zero, subnormal
        hi = sgn;
        lo = 0u;
    }
    return f64_from(hi, lo);
}

// binary64 -> binary32, rounded to nearest, ties to even
__host__ __device__ __forceinline__ float f64_to_f32_bits(double d)
{
    const uint64_t b = f64_bits(d);
    const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
    const uint64_t a = b & 0x7FFFFFFFFFFFFFFFull;
    // keep the exponent and the top 23 fraction bits, the 29 dropped bits rounded to nearest
    // even: adding 2^28 - 1 plus the lowest kept bit carries exactly when the dropped part is
    // above one half, or equal to it with the kept part odd (a carry out of the fraction raises
    // the exponent, as it must)
    const uint64_t r = (a + 0x0FFFFFFFull + ((a >> 29) & 1ull)) >> 29;
    uint32_t out = sgn | (uint32_t)(r - (896ull << 23));         // exponent rebiased 1023 -> 127
    if (r >= (1151ull << 23)) out = sgn | 0x7F800000u;            // beyond the largest float: inf
    if (r < (897ull << 23)) out = sgn;                            // below the smallest normal
    if (a > 0x7FF0000000000000ull) out = sgn | 0x7FC00000u;       // NaN
    return f32_from(out);
}

}  // namespace tkf
