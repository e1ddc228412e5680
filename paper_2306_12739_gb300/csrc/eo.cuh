// Parity blocks of the y-operators (the fused stage in parity blocks, k_spec.cu,
// and the step-by-step forcing and implicit apply in parity blocks,
// k_step_eo.cu).  On the symmetric Chebyshev grid y_j = -y_{Ny-1-j} a
// centro-symmetric operator (M - I, P of both fields, D2) maps the even part
// x_e[i] = x[i] + x[Ny-1-i] to the even part and the odd part x_o[i] = x[i] -
// x[Ny-1-i] to the odd part (i < Ny/2; the centre row of odd Ny alone in x_e),
// and the anti-centro-symmetric D1 maps odd to even and even to odd; y[i] =
// (y_e[i] + y_o[i]) / 2, y[Ny-1-i] = (y_e[i] - y_o[i]) / 2.  A matrix is stored
// as the block of its even output rows [KE][RP2] then the block of its odd
// output rows [KO][RP2], transposed (k-major) and row-padded (spec_eo_image).
#pragma once
#include "dns_internal.hpp"
#include "cvt.cuh"
#include "ff.cuh"

namespace dnsk {
namespace spc {

__host__ __device__ inline int eo_ne(int ny) { return (ny + 1) / 2; }
__host__ __device__ inline int eo_rp(int ny) { return 2 * ((eo_ne(ny) + 1) / 2); }
// floats of one matrix in parity blocks (a multiple of 4: 16-byte copies)
__host__ __device__ inline size_t eo_mat(int ny) { return ((size_t)ny * eo_rp(ny) + 3) / 4 * 4; }

// float-float product of one pair-row p (phase 4 with D2FF): centro-symmetric D2
// (hi part B, residual BL) in parity blocks with the even and odd parts of v
// (hi XH, lo XL); sums (hi, lo) per output row and re/im
__device__ __forceinline__ void eo1ff(const float* B, const float* BL, int NE, int NO, int RP2, const float* XH,
                                      const float* XL, int VS, int p, int c2, float (&eh)[2], float (&el)[2],
                                      float (&oh)[2], float (&ol)[2]) {
    eh[0] = eh[1] = el[0] = el[1] = oh[0] = oh[1] = ol[0] = ol[1] = 0.f;
#pragma unroll 2
    for (int k = 0; k < NE; ++k) {
        const float b = B[k * RP2 + p], bl = BL[k * RP2 + p];
        const float2 x = *(const float2*)&XH[k * VS + c2];
        const float2 xl = *(const float2*)&XL[k * VS + c2];
        ff_add_prod2(eh[0], el[0], b, x.x, bl, xl.x);
        ff_add_prod2(eh[1], el[1], b, x.y, bl, xl.y);
    }
    const size_t ob = (size_t)NE * RP2;
#pragma unroll 2
    for (int k = 0; k < NO; ++k) {
        const float b = B[ob + k * RP2 + p], bl = BL[ob + k * RP2 + p];
        const float2 x = *(const float2*)&XH[(NE + k) * VS + c2];
        const float2 xl = *(const float2*)&XL[(NE + k) * VS + c2];
        ff_add_prod2(oh[0], ol[0], b, x.x, bl, xl.x);
        ff_add_prod2(oh[1], ol[1], b, x.y, bl, xl.y);
    }
}

// Two pair-rows p0, p0 + 1 x one complex column (c2 its real column) of a
// matrix in parity blocks B: the block of the even output rows [KE][RP2]
// contracts XE, the block of the odd output rows [KO][RP2] (after it)
// contracts XO.
__device__ __forceinline__ void eo2(const float* B, int KE, int KO, int RP2, const float* XE, const float* XO, int VS,
                                    int p0, int c2, float (&ye)[2][2], float (&yo)[2][2]) {
#pragma unroll
    for (int r = 0; r < 2; ++r) { ye[r][0] = ye[r][1] = yo[r][0] = yo[r][1] = 0.f; }
#pragma unroll 4
    for (int k = 0; k < KE; ++k) {
        const float2 b = *(const float2*)&B[k * RP2 + p0];
        const float2 x = *(const float2*)&XE[k * VS + c2];
        ye[0][0] += b.x * x.x; ye[0][1] += b.x * x.y; ye[1][0] += b.y * x.x; ye[1][1] += b.y * x.y;
    }
    const float* BO = B + KE * RP2;
#pragma unroll 4
    for (int k = 0; k < KO; ++k) {
        const float2 b = *(const float2*)&BO[k * RP2 + p0];
        const float2 x = *(const float2*)&XO[k * VS + c2];
        yo[0][0] += b.x * x.x; yo[0][1] += b.x * x.y; yo[1][0] += b.y * x.x; yo[1][1] += b.y * x.y;
    }
}

// Two matrices A, B in parity blocks, the same pair-rows and column, with
// their own inputs (the implicit apply of eta: (M - I) x + P G~)
__device__ __forceinline__ void eo2x2(const float* A, const float* B, int KE, int KO, int RP2, const float* XAE,
                                      const float* XAO, const float* XBE, const float* XBO, int VS, int p0, int c2,
                                      bool needA, float (&ae)[2][2], float (&ao)[2][2], float (&be)[2][2],
                                      float (&bo)[2][2]) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) ae[r][c] = ao[r][c] = be[r][c] = bo[r][c] = 0.f;
#pragma unroll 4
    for (int k = 0; k < KE; ++k) {
        const float2 bb = *(const float2*)&B[k * RP2 + p0];
        const float2 xb = *(const float2*)&XBE[k * VS + c2];
        be[0][0] += bb.x * xb.x; be[0][1] += bb.x * xb.y; be[1][0] += bb.y * xb.x; be[1][1] += bb.y * xb.y;
        if (needA) {
            const float2 aa = *(const float2*)&A[k * RP2 + p0];
            const float2 xa = *(const float2*)&XAE[k * VS + c2];
            ae[0][0] += aa.x * xa.x; ae[0][1] += aa.x * xa.y; ae[1][0] += aa.y * xa.x; ae[1][1] += aa.y * xa.y;
        }
    }
    const float* AO = A + KE * RP2;
    const float* BO = B + KE * RP2;
#pragma unroll 4
    for (int k = 0; k < KO; ++k) {
        const float2 bb = *(const float2*)&BO[k * RP2 + p0];
        const float2 xb = *(const float2*)&XBO[k * VS + c2];
        bo[0][0] += bb.x * xb.x; bo[0][1] += bb.x * xb.y; bo[1][0] += bb.y * xb.x; bo[1][1] += bb.y * xb.y;
        if (needA) {
            const float2 aa = *(const float2*)&AO[k * RP2 + p0];
            const float2 xa = *(const float2*)&XAO[k * VS + c2];
            ao[0][0] += aa.x * xa.x; ao[0][1] += aa.x * xa.y; ao[1][0] += aa.y * xa.x; ao[1][1] += aa.y * xa.y;
        }
    }
}

// one pair-row p (phase 4: every thread one pair-row of one column)
__device__ __forceinline__ void eo1(const float* B, int KE, int KO, int RP2, const float* XE, const float* XO, int VS,
                                    int p, int c2, float (&ye)[2], float (&yo)[2]) {
    ye[0] = ye[1] = yo[0] = yo[1] = 0.f;
#pragma unroll 4
    for (int k = 0; k < KE; ++k) {
        const float b = B[k * RP2 + p];
        const float2 x = *(const float2*)&XE[k * VS + c2];
        ye[0] += b * x.x; ye[1] += b * x.y;
    }
    const float* BO = B + KE * RP2;
#pragma unroll 4
    for (int k = 0; k < KO; ++k) {
        const float b = BO[k * RP2 + p];
        const float2 x = *(const float2*)&XO[k * VS + c2];
        yo[0] += b * x.x; yo[1] += b * x.y;
    }
}

// natural rows of pair-row p: y0 = p and, below the centre, y1 = Ny-1-p
struct EoRows {
    int y0, y1;
    bool pair;
};
__device__ __forceinline__ EoRows eo_rows(int p, int Ny) {
    EoRows r;
    r.y0 = p;
    r.y1 = Ny - 1 - p;
    r.pair = p < Ny / 2;
    return r;
}

// The even and odd parts of two FP64 values as float-float pairs (h, l), from
// their single-precision splits (x = h + l to 2^-48): a TwoSum (Knuth) of the
// high parts, the low parts added to its error; the FP64 pipe is not used.
__device__ __forceinline__ void eo_ff(double x0, double x1, float& eh, float& el, float& oh, float& ol) {
    const float h0 = d2f(x0), h1 = d2f(x1);
    const float l0 = d2f(x0 - f2d(h0)), l1 = d2f(x1 - f2d(h1));
    float s = h0 + h1, bb = s - h0;
    eh = s;
    el = ((h0 - (s - bb)) + (h1 - bb)) + (l0 + l1);
    s = h0 - h1;
    bb = s - h0;
    oh = s;
    ol = ((h0 - (s - bb)) + (-h1 - bb)) + (l0 - l1);
}

// MINB: CTAs per SM the registers are budgeted for (2, or 3 at 80 registers;
// shared memory allows 3): chosen by timing whole steps

}  // namespace spc
}  // namespace dnsk
