// IEEE 754 binary32 <-> binary64 conversions done with integer operations.
//
// On GB300 the FP64 pipe is the scarce resource of the FP64 residual kernel; these
// conversions move the format changes of the mixed-precision path (the complex64
// correction into the complex128 iterate, the complex128 residual into the complex64
// right-hand side) onto the integer pipes.  Written from the binary32 / binary64
// layouts of IEEE 754-2008 (sign, biased exponent, fraction; bias 127 / 1023) and its
// roundTiesToEven rule.  Zero, infinities and NaNs are kept; binary32 subnormals
// (magnitudes below 2^-126 ~ 1.2e-38) are flushed to a signed zero in both directions.
#pragma once
#include <cuda_runtime.h>

namespace helm {

// exact widening: exponent rebias by 1023 - 127 = 896, fraction shifted up by 29 bits
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned mag = b & 0x7fffffffu;
    unsigned hi, lo;
    if (mag < 0x00800000u) {             // zero or subnormal
        hi = sign;
        lo = 0u;
    } else if (mag >= 0x7f800000u) {     // infinity or NaN
        hi = sign | 0x7ff00000u | ((mag & 0x007fffffu) >> 3);
        lo = mag << 29;
    } else {
        hi = sign | ((mag >> 3) + (896u << 20));
        lo = mag << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// narrowing with round-to-nearest, ties to even
__device__ __forceinline__ float d2f_bits(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) {                                       // infinity or NaN
        const bool nan = ((hi & 0x000fffffu) | lo) != 0u;
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x00400000u : 0u));
    }
    const int E = e - 896;
    if (E >= 255) return __uint_as_float(sign | 0x7f800000u);   // overflow
    if (E <= 0) return __uint_as_float(sign);                   // below the normal range
    const unsigned m = ((hi & 0x000fffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    unsigned v = ((unsigned)E << 23) + m;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) v += 1u;  // carry may bump E
    return __uint_as_float(sign | v);
}

}  // namespace helm
