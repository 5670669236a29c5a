// bits.cuh -- conversions between FP64 and FP32 and magnitude comparisons
// done on the IEEE 754 bit patterns with integer operations.  On GB300 the
// FP64<->FP32 conversion instructions and FP64 min/max issue on the FP64
// pipe, 1/64 of the FP32 rate, which the FP64-bound kernels cannot spare.
//
// Header-only, usable from device and host code (host: plain C++, so that
// the functions are checked on the CPU against the host's own conversions).
#pragma once

#include <stdint.h>
#include <string.h>

#if !defined(__CUDACC__)
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace elder {

__host__ __device__ __forceinline__ uint32_t bits_of(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
#endif
}

__host__ __device__ __forceinline__ float float_of(uint32_t u)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, 4);
    return x;
#endif
}

__host__ __device__ __forceinline__ uint64_t bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

__host__ __device__ __forceinline__ double double_of(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

// FP32 value of an FP64 number: the exponent rebiased by 127 - 1023, the top
// 23 of the 52 mantissa bits kept (truncated toward zero, not rounded);
// magnitudes below 2^-126 become a zero of the same sign, those from 2^128 up
// (and NaN) infinity.  For the residual's round-off scale, a magnitude needed
// to a few digits, and for powers of two, which it converts exactly.
__host__ __device__ __forceinline__ float d2f_trunc(double x)
{
    const uint64_t u = bits_of(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const uint32_t sign = hi & 0x80000000u;
    uint32_t bits = sign | ((uint32_t)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    bits = e <= 896 ? sign : (e >= 1151 ? (sign | 0x7F800000u) : bits);
    return float_of(bits);
}

// FP64 value of an FP32 number, exact like the conversion instruction:
// exponent rebiased by 1023 - 127, mantissa shifted up by 29 bits; signed
// zeros in the integer path, subnormals, infinities and NaN by the
// conversion itself.
__host__ __device__ __forceinline__ double f2d_exact(float x)
{
    const uint32_t u = bits_of(x), a = u & 0x7FFFFFFFu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (a == 0u) return double_of(sign);
    if (a < 0x00800000u || a >= 0x7F800000u) return (double)x;
    return double_of(sign | (((uint64_t)a + (896ull << 23)) << 29));
}

// |x| as its bit pattern, which orders like the magnitude; NaN maps to the
// pattern of +inf
__host__ __device__ __forceinline__ uint32_t mag_bits(float x)
{
    const uint32_t a = bits_of(x) & 0x7FFFFFFFu;
    return a > 0x7F800000u ? 0x7F800000u : a;
}

}  // namespace elder
