// binary64 <-> binary32 conversions on integer operations, from the IEEE 754
// interchange formats (sign, biased exponent 11 / 8 bits, fraction 52 / 23
// bits).  On this GPU the hardware conversions issue to the FP64 pipe, which
// is far slower than the integer and FP32 pipes; the mixed-precision kernels
// convert their FP64 state with these instead.
//
// d2f: round to nearest, ties to even.  Magnitudes below the smallest normal
//      binary32 (2^-126) give a signed zero (no subnormal results); overflow
//      gives infinity, NaN stays NaN.
// f2d: exact for normal binary32 values and zeros; binary32 subnormals give a
//      signed zero; infinity and NaN are kept.
#pragma once
#include <cuda_runtime.h>

namespace dnsk {

__host__ __device__ __forceinline__ unsigned d2f_bits(unsigned hi, unsigned lo) {
    const unsigned s = hi & 0x80000000u, ah = hi & 0x7fffffffu;
    // exponent rebias 1023 -> 127 (896 << 20 in the high word) and the leading
    // 23 fraction bits; the 29 dropped bits decide the rounding
    unsigned f = ((ah - 0x38000000u) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
    if (ah < 0x38100000u) f = 0u;                 // below 2^-126
    if (ah >= 0x47f00000u)                        // 2^128 and beyond, infinity, NaN
        f = (ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
    return s | f;
}

__host__ __device__ __forceinline__ void f2d_bits(unsigned f, unsigned* hi, unsigned* lo) {
    const unsigned s = f & 0x80000000u, af = f & 0x7fffffffu;
    unsigned h = s | ((af >> 3) + 0x38000000u), l = af << 29;
    if (af < 0x00800000u) { h = s; l = 0u; }      // zero or subnormal
    if (af >= 0x7f800000u) { h = s | 0x7ff00000u | ((af & 0x007fffffu) ? 0x00080000u : 0u); l = 0u; }
    *hi = h;
    *lo = l;
}

#ifdef __CUDACC__
__device__ __forceinline__ float d2f(double x) {
    return __uint_as_float(d2f_bits((unsigned)__double2hiint(x), (unsigned)__double2loint(x)));
}

__device__ __forceinline__ double f2d(float x) {
    unsigned hi, lo;
    f2d_bits(__float_as_uint(x), &hi, &lo);
    return __hiloint2double((int)hi, (int)lo);
}
#endif

}  // namespace dnsk
