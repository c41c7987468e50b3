// Exact float <-> double conversions built from 32-bit integer operations.
//
// The single-precision states (CDBM_FP32_BULK) convert every stored deviation to
// double for the conserved sums and round every equilibrium value back to float:
// 32 conversions per cell and Runge-Kutta stage.  On GB300 the conversion
// instructions issue on the FP64 pipe, the scarce unit of that path, while the
// integer pipes are nearly idle.  So the common cases are done on the bit patterns:
//
//   float -> double (exact): a normal float with magnitude bits m (8 exponent and
//     23 fraction bits) has the double high word (m >> 3) + ((1023 - 127) << 20)
//     and low word m << 29; zero keeps its sign;
//   double -> float (IEEE round to nearest, ties to even): for a result with a
//     normal float exponent, the 23 leading fraction bits are kept and the 29
//     dropped ones decide the rounding increment, whose carry may run into the
//     exponent (and to infinity past the largest float, as the IEEE rule says).
//
// Subnormal, infinite and NaN operands, and results outside the normal float range
// other than zero, are left to the conversion instruction in an out-of-line call,
// which the states of this method never reach.  The same source compiles for the
// host, where a unit test checks it against the C conversions bit for bit.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define CDBM_CVT_HD __host__ __device__ __forceinline__
#define CDBM_CVT_RARE static __host__ __device__ __noinline__
#else
#define CDBM_CVT_HD inline
#define CDBM_CVT_RARE static inline
#endif

namespace cdbm {

CDBM_CVT_HD uint32_t f32_bits(float v)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(v);
#else
    uint32_t b;
    std::memcpy(&b, &v, sizeof b);
    return b;
#endif
}

CDBM_CVT_HD float f32_from_bits(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float v;
    std::memcpy(&v, &b, sizeof v);
    return v;
#endif
}

CDBM_CVT_HD uint32_t f64_hi(double v)
{
#if defined(__CUDA_ARCH__)
    return (uint32_t)__double2hiint(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    return (uint32_t)(b >> 32);
#endif
}

CDBM_CVT_HD uint32_t f64_lo(double v)
{
#if defined(__CUDA_ARCH__)
    return (uint32_t)__double2loint(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    return (uint32_t)b;
#endif
}

CDBM_CVT_HD double f64_from_words(uint32_t hi, uint32_t lo)
{
#if defined(__CUDA_ARCH__)
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t b = ((uint64_t)hi << 32) | lo;
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
#endif
}

CDBM_CVT_RARE double widen_rare(float v) { return (double)v; }
CDBM_CVT_RARE float narrow_rare(double v) { return (float)v; }

// (double)v, exactly.
CDBM_CVT_HD double widen_f32(float v)
{
    const uint32_t b = f32_bits(v), s = b & 0x80000000u, m = b & 0x7fffffffu;
    if (m - 0x00800000u >= 0x7f000000u && m != 0u) return widen_rare(v);   // subnormal, inf, NaN
    return f64_from_words(s | (m != 0u ? (m >> 3) + 0x38000000u : 0u), m << 29);
}

// (float)v with round to nearest, ties to even.
CDBM_CVT_HD float narrow_f64(double v)
{
    const uint32_t hi = f64_hi(v), lo = f64_lo(v);
    const uint32_t s = hi & 0x80000000u, mh = hi & 0x7fffffffu;
    if ((mh >> 20) - 897u < 254u) {                   // float exponent 1..254 before rounding
        uint32_t t = ((mh - (896u << 20)) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;        // the 29 dropped fraction bits
        t += (uint32_t)(rest > 0x10000000u) | ((uint32_t)(rest == 0x10000000u) & t);
        return f32_from_bits(s | t);
    }
    if (mh == 0u) return f32_from_bits(s);            // zero, or below every float: signed zero
    return narrow_rare(v);
}

}  // namespace cdbm

#undef CDBM_CVT_HD
#undef CDBM_CVT_RARE
