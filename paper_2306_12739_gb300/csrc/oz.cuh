// Exact tensor-core digit product (Ozaki et al. 2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", with small integers in place of floating slices): the
// pieces shared by the D2 v kernel (k_d2v_tc.cu) and the fused per-wavenumber
// stage (k_spec.cu), which run the same digit arithmetic and so produce the
// same bits.  A value x with |x| < 2^f is written as NDIG signed 7-bit digits
// of x 2^-f; digits are integers of magnitude <= 127, exact in BF16, and a
// level L = s + t of digit products (digit s of one operand, t of the other)
// summed over K <= 64 stays below 2^24: the FP32 accumulators of
// tcgen05.mma.kind::f16 hold every level exactly.  Also: the shared-memory
// descriptors (no swizzle, K-major core matrices), the instruction descriptor,
// the MMA and TMEM loads, and the Horner combination of the levels.
#pragma once
#include <cstdint>
#include "ff.cuh"
#include "mbar.cuh"

namespace dnsk {
namespace oz {

constexpr int NDIG = 6;            // digits per value (7 bits each: 42 fraction bits)
constexpr int NLEV = 6;            // levels s + t kept
constexpr int FBITS = 7 * NDIG;
constexpr int MROWS = 128;          // MMA M: 64 rows of D2 used, the rest never read back

// one digit slice of D2's image: 64 rows x KP, BF16 (bytes)
__host__ __device__ inline size_t slice_a(int KP) { return (size_t)64 * KP * 2; }

// shared-memory matrix descriptor, no swizzle, K-major core matrices (8 rows x
// 16 bytes): LBO between core matrices along K, SBO between 8-row groups
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D F32, A = B = BF16, both K-major
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// biased binary exponent of |x| (0 for zero and subnormals)
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// The NDIG digits of x in units of 2^f (|x| < 2^f), as BF16 bit patterns:
// the magnitude rounded to FBITS fraction bits, 7 bits per digit, the sign on
// every digit.  Integer operations only.
__device__ __forceinline__ void digits(double x, int f, unsigned short (&d)[NDIG]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long X = 0;
    if (ex > 0) {
        const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int rs = 1075 - FBITS + f - ex;   // right shift: X = round(m 2^(ex - 1075 + FBITS - f))
        if (rs < 64) X = rs > 0 ? (m + (1ull << (rs - 1))) >> rs : m;
        if (X >= (1ull << FBITS)) X = (1ull << FBITS) - 1;
    }
    const unsigned short sg = (bits >> 63) ? 0x8000u : 0u;
    const unsigned hi = (unsigned)(X >> 21), lo = (unsigned)X & 0x1FFFFFu;   // digits 0..2 | 3..5
    static_assert(NDIG == 6, "the split into two 21-bit halves assumes six digits");
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
        const unsigned u = (s < 3 ? hi >> (7 * (2 - s)) : lo >> (7 * (5 - s))) & 127u;
        // the BF16 of a small integer u: the float u (exact), its top 16 bits
        const float fu = __int_as_float(0x4B000000 | (int)u) - 8388608.0f;
        d[s] = u ? (unsigned short)((unsigned)__float_as_int(fu) >> 16) | sg : (unsigned short)0;
    }
}

// 2^n as a float (0 below the normal range)
__device__ __forceinline__ float p2f(int n) {
    if (n < -126) return 0.f;
    if (n > 127) n = 127;
    return __int_as_float((n + 127) << 23);
}

__device__ __forceinline__ void ld8(unsigned taddr, float* v) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Horner over the levels from the smallest, (hi, lo) = acc_L + 2^-7 (hi, lo),
// for W consecutive accumulator columns of this thread's TMEM lane; level L
// starts at column L * lstride.  Returns the float-float sums in hi, lo.
template <int W>
__device__ __forceinline__ void combine_levels(unsigned taddr, int lstride, float (&hi)[W], float (&lo)[W]) {
    static_assert(W == 8 || W == 16, "TMEM loads of 8 or 16 columns");
    float a[W];
#pragma unroll
    for (int i = 0; i < W; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
    for (int L = NLEV - 1; L >= 0; --L) {
        if (W == 16) ld16(taddr + (unsigned)(L * lstride), a);
        else ld8(taddr + (unsigned)(L * lstride), a);
#pragma unroll
        for (int i = 0; i < W; ++i) {
            hi[i] *= 0.0078125f;
            lo[i] *= 0.0078125f;
            ff_add(hi[i], lo[i], a[i], 0.f);
        }
    }
}

}  // namespace oz
}  // namespace dnsk
