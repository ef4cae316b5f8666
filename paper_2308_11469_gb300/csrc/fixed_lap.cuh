// Laplacian numerators of FP64 values summed exactly in 64-bit fixed point.
//
// The FP64 residual r = f - (Delta_h + k^2) u (Section 2.4's FD system, formed every outer
// step) needs, per node and component, the sum of the 2D neighbours minus 2D times the
// node: terms of size ~ (2D/h^2)|u| cancelling down to |r|.  Evaluated in FP64 that sum
// costs 2D - 1 additions on the FP64 pipe, which GB300 runs at a small fraction of its
// integer rate, and each addition rounds.  Here the values a residual tile reads are put
// on one 64-bit fixed-point scale set by the largest binary exponent among them (each
// value v becomes trunc(v * 2^(1080 - emax)): exact for every value within a factor 32 of
// the largest, the others truncated below 2^-57 of it), the numerator is summed exactly
// with integer additions, and rounded once to FP64 (round to nearest, ties to even).  The
// result is at least as accurate as the FP64 evaluation, whose additions each round at
// half an ulp of the partial sums.
//
// Written from the binary64 layout of IEEE 754-2008 (sign bit, 11-bit biased exponent,
// 52-bit fraction with an implicit leading 1 for normal numbers; bias 1023) and its
// roundTiesToEven rule.  The scale exponent is raised to at least FX_EMIN (values below
// 2^-959 then round to multiples of 2^-1016, far below any residual they could change); a
// tile holding a value above 2^1007, an infinity or a NaN has no fixed-point scale and its
// residuals are NaN (the FP64 evaluation would overflow there too), which the status rule
// reports as non-finite.
#pragma once
#include <cuda_runtime.h>
#include <cstring>

namespace helm {

// bit pattern of v and leading-zero count of a 64-bit word, on the device and the host
// (the host form lets the arithmetic be checked against exact rationals on a CPU)
__host__ __device__ __forceinline__ unsigned long long fx_bits(double v)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    std::memcpy(&b, &v, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double fx_from_bits(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
#endif
}

__host__ __device__ __forceinline__ int fx_clz(unsigned long long a)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

constexpr int FX_EMIN = 64;
constexpr int FX_EMAX = 2030;

// NaN of the non-representable tiles
__host__ __device__ __forceinline__ double fx_nan() { return fx_from_bits(0x7ff8000000000000ull); }

// biased exponent field of v (0: zero or subnormal; 2047: infinity or NaN)
__host__ __device__ __forceinline__ int fx_exp(double v)
{
    return (int)((unsigned)(fx_bits(v) >> 52) & 0x7ffu);
}

// trunc(v * 2^(1080 - emax)) for fx_exp(v) <= emax: |result| < 2^58.  Zero and subnormal
// inputs give 0.
__host__ __device__ __forceinline__ long long fx_fix(double v, int emax)
{
    const unsigned long long b = fx_bits(v);
    const int e = (int)((b >> 52) & 0x7ffull);
    // significand with its leading 1 at bit 62: v = m * 2^(e - 1085)
    const unsigned long long m = ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) << 10;
    const int s = emax - e + 5;                       // >= 5
    const unsigned long long a = (e != 0 && (unsigned)s < 64u) ? (m >> s) : 0ull;
    const long long sg = (long long)b >> 63;          // 0 or -1
    return ((long long)a ^ sg) - sg;
}

// L * 2^(emax - 1080) rounded to the nearest binary64, ties to even.  Needs |L| < 2^62
// and FX_EMIN <= emax <= FX_EMAX (the result is then normal and finite, or zero).
__host__ __device__ __forceinline__ double fx_to_double(long long L, int emax)
{
    const unsigned long long sign = (unsigned long long)L & 0x8000000000000000ull;
    const unsigned long long a = (unsigned long long)(L < 0 ? -L : L);
    const int lz = fx_clz(a);                         // 64 when a == 0
    const unsigned long long nrm = a << (lz & 63);    // leading 1 at bit 63
    unsigned long long q = nrm >> 11;                 // 53-bit significand, leading 1 at bit 52
    const unsigned long long rest = nrm & 0x7ffull;   // the 11 bits rounded away
    q += (rest > 0x400ull || (rest == 0x400ull && (q & 1ull))) ? 1ull : 0ull;
    // value = q * 2^(emax - 1069 - lz): biased exponent emax + 6 - lz.  Adding q (bit 52
    // set) to the field (exponent - 1) supplies the leading 1, and a rounding carry into
    // bit 53 raises the exponent by one with a zero fraction.
    const unsigned long long mag = ((unsigned long long)(emax + 5 - lz) << 52) + q;
    return (a == 0ull) ? 0.0 : fx_from_bits(sign | mag);
}

}  // namespace helm
