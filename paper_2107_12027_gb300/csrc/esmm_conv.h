// esmm_conv.h -- FP64 <-> FP32 conversions in integer arithmetic.
//
// On this GPU a hardware conversion between double and float issues on the
// FP64 pipe, the scarcest unit (1/64 of the FP32 rate).  The node pass and
// the update kernel of the mixed form convert a dozen values per node, next
// to FP64 arithmetic that keeps that pipe busy; these functions do the same
// conversions on the integer pipes instead, bit for bit equal to the IEEE 754
// conversions (round to nearest, ties to even, for the narrowing one).  The
// exponent and fraction fields are moved between the formats directly; the
// cases outside the common path (results that are subnormal, overflow, an
// infinity or NaN operand) fall back to the hardware conversion.
//
// Host and device code share these definitions; the host build is what the
// CPU tests check against the compiler's own casts.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define ESMM_CONV_HD __host__ __device__ __forceinline__
#else
#define ESMM_CONV_HD static inline
#endif

namespace esmm {

ESMM_CONV_HD uint64_t conv_bits64(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

ESMM_CONV_HD double conv_double(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

ESMM_CONV_HD uint32_t conv_bits32(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

ESMM_CONV_HD float conv_float(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// x rounded to the nearest float, ties to even.  A double with biased
// exponent e in [897, 1150] has a normal float of biased exponent e - 896
// as its truncation: keep the top 23 of its 52 fraction bits and round on
// the 29 dropped ones (a carry out of the fraction steps the exponent, and
// out of the largest finite float gives infinity, as rounding does).
ESMM_CONV_HD float d2f_int(double x)
{
    const uint64_t b = conv_bits64(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u <= 253u) {
        const uint64_t m = b & 0x000fffffffffffffull;
        uint32_t r = ((e - 896u) << 23) | (uint32_t)(m >> 29);
        const uint32_t rem = (uint32_t)m & 0x1fffffffu;
        r += (uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & (r & 1u));
        return conv_float(r | sign);
    }
    if ((b << 1) == 0) return conv_float(sign);   // +-0
    return (float)x;
}

// the double equal to x (exact): a normal float's biased exponent e maps to
// e + 896 and its 23 fraction bits to the top of the 52
ESMM_CONV_HD double f2d_int(float x)
{
    const uint32_t u = conv_bits32(x);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    if (e - 1u < 254u)
        return conv_double(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
    if ((u << 1) == 0) return conv_double(sign);   // +-0
    return (double)x;
}

}  // namespace esmm
