// Fused per-wavenumber stage of the mixed path: everything of one sub-step
// that follows the physical-space stage, in one launch (paper Sec. 3.1-3.2):
//   forcing     F = -k^2 Nv - D1 (i kx Nu + i kz Nw),  G = i kz Nu - i kx Nw
//               (Eqs. Dv, eta) and the RK3 combination F~, G~ of the sub-step;
//   implicit    x+ = x_t + ((M_h - I) x_t + P_h F~)  per wavenumber pair
//   apply       (increment form of Eqs. CN1, CN2; the increment in single
//               precision, one double add);
//   derivatives Dv, D2v, D eta of the new state, written in the per-plane
//               layout the next physical-space stage reads (so the next
//               sub-step, or the next step, starts with the transforms);
//   mean flow   the rows of the mean-flow update (Eqs. CN3, CN4) in leading
//               CTAs, the last of a member's row CTAs finishing it (constant-
//               flux gamma, profiles, RK accumulators of <uv>, <wv>).
// One CTA per (wavenumber pair (n, |m|), member chunk): both modes +-m and
// both fields.  The pair's four operators and D1 arrive by TMA bulk copies (the
// third sub-step needs only the P matrices); D2 and its residual are copied
// over the eta operators once those are used.  The CTA's 256 threads run the
// stages in four phases separated by barriers; in the two middle phases the
// two halves of the CTA work on v and eta side by side.
//
// D2 v needs more than single precision: the collocation D2 has entries up to
// ~N^4/10 that cancel in every row, so a single-precision sum (or any FP32-
// accumulated split tensor-core product) loses ~1e-5 of |D2 v|.  Where Ny <= 64
// the tensor-core digit kernel (k_d2v_tc.cu, exact accumulation) computes it
// from the new FP64 state after this launch; otherwise this kernel sums it in
// float-float: D2 and v are held as pairs of single-precision numbers and every
// product enters a compensated sum (TwoSum, the FMA product residual, the cross
// terms into the low part).
//
// With d2fuse the stage runs that digit product itself (oz.cuh, the same digit
// arithmetic, so the same bits): the image of D2's digits is copied over the
// operators phase 2 has finished with while phase 3 runs, the new state's
// digits go over P_v after phase 3, one thread issues the MMAs while the CTA
// computes D v, and four warps read the six levels back from TMEM.  A sub-step
// is then two launches per member block (plane stage, this one).
#include "dns_internal.hpp"
#include "mbar.cuh"
#include "cvt.cuh"
#include "ff.cuh"
#include "mean.cuh"
#include "oz.cuh"
#include "eo.cuh"

namespace dnsk {

namespace spc {

constexpr int THREADS = 256;
constexpr int HALF = THREADS / 2;
constexpr int NCR_MAX = 32;   // real columns per CTA (modes x members x re/im)

constexpr int DCOL = 16;      // real columns of the fused D2 v digit product (MMA N)
constexpr unsigned DTCOLS = 128;   // its TMEM columns: NLEV x DCOL = 96, allocated as 128

// Member chunk: at most NCR_MAX real columns per CTA (two modes, re and im);
// with the fused D2 v at most DCOL.
__host__ __device__ inline int chunk_members(const GroupView& g) {
    const int cap = g.d2fuse ? DCOL / 4 : NCR_MAX / 4;
    const int ec = (g.spec_ec > 0 && g.spec_ec <= cap) ? g.spec_ec : cap;
    return g.E < ec ? g.E : ec;
}
__host__ __device__ inline int chunks(const GroupView& g) {
    const int ec = chunk_members(g);
    return (g.E + ec - 1) / ec;
}
// row stride (floats) of the shared-memory vectors: the chunk's real columns
__host__ __device__ inline int vec_stride(const GroupView& g) { return 4 * chunk_members(g); }
__host__ __device__ inline size_t vec_floats(const GroupView& g) { return (size_t)g.ny * vec_stride(g); }
// Operator slot (floats): one [Ny][RP] matrix; with the fused D2 v at least
// two digit slices of D2's image (2 x 64 rows x KP BF16 = 64 KP floats).
__host__ __device__ inline size_t slot_floats(const GroupView& g) {
    const size_t m = (size_t)g.ny * g.rp, s2 = (size_t)64 * g.kp;
    return (g.d2fuse && s2 > m) ? s2 : m;
}
// shared memory: 4 operator slots (the eta pair reused for D2 and its residual
// after phase 2; with d2fuse the image of D2's digits in slots 0, 2, 3 from
// phase 3 and the new state's digits in slot 1 in phase 4) | D1 [Ny][RP] |
// 7 vectors [Ny][vec_stride] | 4 mbarriers
__host__ __device__ inline size_t smem_bytes(const GroupView& g) {
    // (with d2fuse, 128 more bytes after the mbarriers: column exponents, TMEM base, status)
    const size_t b = (4 * slot_floats(g) + (size_t)g.ny * g.rp + 7 * vec_floats(g)) * sizeof(float) + 32 +
                     (g.d2fuse ? 128 : 0);
    // with d2fuse, room for the 64 unused A rows that follow the last digit slice
    const size_t t = g.d2fuse ? 3 * slot_floats(g) * sizeof(float) + 3 * (size_t)64 * g.kp * 2 : 0;
    return b > t ? b : t;
}
// With d2fuse the MMA's A operand is M = 128 rows of which 64 are D2's: the
// other 64 read the 128 KP bytes that follow each slice (never read back), so
// those must lie inside the CTA's shared memory, also after the last slice.
__host__ __device__ inline bool fused_d2_fits(const GroupView& g) {
    const size_t slot = slot_floats(g) * sizeof(float), sa = (size_t)64 * g.kp * 2;
    return 3 * slot + 3 * sa <= smem_bytes(g) && 6 * (size_t)DCOL * g.kp * 2 <= slot;
}

__device__ __forceinline__ void bulk(void* dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Finish of a member's mean-flow update after its last row CTA (see
// mean_finish): gamma, the profiles, the RK accumulators of <uv>, <wv>.  The
// pre-gamma rows dU, dW were written by other CTAs of this launch: they are
// read through L2.
__device__ void finish_member(const GroupView& g, int s, int e, unsigned char* sm) {
    const int Ny = g.ny, My = g.my;
    double* red = (double*)sm;
    const int hi = (s == 0) ? 0 : 1;
    const double* Ug = g.mops[hi] + 2 * (size_t)Ny * Ny + 2 * (size_t)Ny;
    const double* Un = g.dU + (size_t)e * My;
    const double* Wn = g.dW + (size_t)e * My;
    const double* Ut = g.U_t + (size_t)e * My;
    const double* Wt = g.W_t + (size_t)e * My;
    double gam = 0.0;
    if (g.flow == 1) {
        double fl = 0.0, fg = 0.0;
        for (int j = threadIdx.x; j < My; j += blockDim.x)
            fl += g.ccw[j] * ((j > 0 && j < My - 1) ? __ldcg(Un + j) : Ut[j]);
        for (int i = threadIdx.x; i < Ny; i += blockDim.x) fg += g.ccw[i + 1] * Ug[i];
        fl = block_sum(fl, red);
        fg = block_sum(fg, red);
        gam = (g.bulk_flux - fl) / fg;
    }
    double* Uo = (s == 2) ? (g.U_t + (size_t)e * My) : (g.U_s + (size_t)e * My);
    double* Wo = (s == 2) ? (g.W_t + (size_t)e * My) : (g.W_s + (size_t)e * My);
    const double u0 = Ut[0], u1 = Ut[My - 1], w0 = Wt[0], w1 = Wt[My - 1];
    __syncthreads();
    for (int j = threadIdx.x; j < My; j += blockDim.x) {
        const bool wall = (j == 0 || j == My - 1);
        Uo[j] = wall ? (j == 0 ? u0 : u1) : __ldcg(Un + j) + gam * Ug[j - 1];
        Wo[j] = wall ? (j == 0 ? w0 : w1) : __ldcg(Wn + j);
        const size_t o = (size_t)e * My + j;
        if (s == 0) {
            g.AU[o] = g.uv[o];
            g.AW[o] = g.wv[o];
        } else if (s == 1) {
            g.AU[o] = (1.0 / 6.0) * g.AU[o] + (4.0 / 6.0) * g.uv[o];
            g.AW[o] = (1.0 / 6.0) * g.AW[o] + (4.0 / 6.0) * g.wv[o];
        }
    }
    if (threadIdx.x == 0) g.gamma[e] = gam;
    // the step is complete: the next step draws new noise
    if (s == 2 && g.fn > 0 && e == 0 && threadIdx.x == 0) *g.fstep += 1ULL;
}

// Rows of the mean-flow update (one warp per interior row), then the member's
// finish by whichever of its row CTAs completes last (a counter per member,
// reset by that CTA for the next launch).
__device__ void mean_cta(const GroupView& g, int s, int b, unsigned char* sm) {
    const int E = g.E, per = (g.ny + 7) / 8;
    const int e = b % E, r = b / E;
    if (!DNS_CK(g.status, r < per, CK_SPEC, b)) return;
    mean_rows(g, s, e, r * (THREADS / 32), sm);
    __shared__ int last;
    __threadfence();        // this CTA's rows are visible device-wide before it counts itself
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&g.mcnt[e], 1) == per - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    finish_member(g, s, e, sm);
    if (threadIdx.x == 0) g.mcnt[e] = 0;
}

// Bounds check of the debug build (a no-op otherwise): the mode, interior
// plane and member of an access, which fix every index of the H and P layouts
__device__ __forceinline__ bool in_range(const GroupView& g, int q, int y, int e) {
    return DNS_CK(g.status, (unsigned)q < (unsigned)g.nmodes && (unsigned)y < (unsigned)g.ny && (unsigned)e < (unsigned)g.E,
                  CK_SPEC, ((long long)q * g.ny + y) * g.E + e);
}

// Columns of a CTA: j = which * ec + el (which 0: mode +m, 1: mode -m; el the
// member in the chunk), real column 2 j + c.
struct Cols {
    int p, n, am, nq, q1, q2, e0, ec, C;
};

__device__ __forceinline__ int col_q(const Cols& c, int j) { return j < c.ec ? c.q1 : c.q2; }
__device__ __forceinline__ int col_e(const Cols& c, int j) { return c.e0 + (j < c.ec ? j : j - c.ec); }

// 4-row x 1-complex-column products of two transposed operators with two
// right-hand sides: a = A x, b = B y (rows r0..r0+3, shared memory operands)
__device__ __forceinline__ void mm2(const float* A, const float* B, const float* X, const float* Y, int Ny, int RP,
                                    int VS, int r0, int c2, bool needA, float (&a)[2][4], float (&b)[2][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) { a[0][i] = a[1][i] = b[0][i] = b[1][i] = 0.f; }
#pragma unroll 4
    for (int k = 0; k < Ny; ++k) {
        const float4 bk = *(const float4*)&B[k * RP + r0];
        const float2 yk = *(const float2*)&Y[k * VS + c2];
        b[0][0] += bk.x * yk.x; b[0][1] += bk.y * yk.x; b[0][2] += bk.z * yk.x; b[0][3] += bk.w * yk.x;
        b[1][0] += bk.x * yk.y; b[1][1] += bk.y * yk.y; b[1][2] += bk.z * yk.y; b[1][3] += bk.w * yk.y;
        if (needA) {
            const float4 ak = *(const float4*)&A[k * RP + r0];
            const float2 xk = *(const float2*)&X[k * VS + c2];
            a[0][0] += ak.x * xk.x; a[0][1] += ak.y * xk.x; a[0][2] += ak.z * xk.x; a[0][3] += ak.w * xk.x;
            a[1][0] += ak.x * xk.y; a[1][1] += ak.y * xk.y; a[1][2] += ak.z * xk.y; a[1][3] += ak.w * xk.y;
        }
    }
}

// 4-row x 1-complex-column product of one transposed operator (shared memory)
// with a right-hand side: a = A x
__device__ __forceinline__ void mm1(const float* A, const float* X, int Ny, int RP, int VS, int r0, int c2,
                                    float (&a)[2][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[0][i] = a[1][i] = 0.f;
#pragma unroll 4
    for (int k = 0; k < Ny; ++k) {
        const float4 ak = *(const float4*)&A[k * RP + r0];
        const float2 xk = *(const float2*)&X[k * VS + c2];
        a[0][0] += ak.x * xk.x; a[0][1] += ak.y * xk.x; a[0][2] += ak.z * xk.x; a[0][3] += ak.w * xk.x;
        a[1][0] += ak.x * xk.y; a[1][1] += ak.y * xk.y; a[1][2] += ak.z * xk.y; a[1][3] += ak.w * xk.y;
    }
}

// 4-row x 1-complex-column product of D1 (transposed [k][RP]) with a
// right-hand side, both in shared memory
__device__ __forceinline__ void d1mm(const float* D1T, const float* X, int Ny, int RP, int VS, int r0, int c2,
                                     float (&a)[2][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[0][i] = a[1][i] = 0.f;
#pragma unroll 4
    for (int k = 0; k < Ny; ++k) {
        const float4 d = *(const float4*)&D1T[k * RP + r0];
        const float2 x = *(const float2*)&X[k * VS + c2];
        a[0][0] += d.x * x.x; a[0][1] += d.y * x.x; a[0][2] += d.z * x.x; a[0][3] += d.w * x.x;
        a[1][0] += d.x * x.y; a[1][1] += d.y * x.y; a[1][2] += d.z * x.y; a[1][3] += d.w * x.y;
    }
}

// Loads of an implicit-apply task, issued before its products so that their
// latency overlaps them: x_t (FP64) and, in the third sub-step, (M_1 - I) x_t.
__device__ __forceinline__ void apply_prefetch(const GroupView& g, int s, int f, const Cols& c, int r0, int j,
                                               double2 (&x)[4], float2 (&m1)[4]) {
    const int Ny = g.ny, E = g.E;
    const int q = col_q(c, j), e = col_e(c, j);
    const double2* X = f == 0 ? g.v_t : g.e_t;
    const float2* M1 = (const float2*)(f == 0 ? g.mx1_v : g.mx1_e);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int y = r0 + i;
        x[i] = make_double2(0.0, 0.0);
        m1[i] = make_float2(0.f, 0.f);
        if (y >= Ny || !in_range(g, q, y, e)) continue;
        const size_t o = ((size_t)q * Ny + y) * E + e;
        x[i] = X[o];
        if (s == 2) m1[i] = M1[o];
    }
}

// The implicit apply of one field for a 4-row x 1-complex-column task, from
// x_t (FP64) and, in the third sub-step, the stored (M_1 - I) x_t, both
// loaded by apply_prefetch before the task's products: writes x+ (FP64; over
// x_t in the third sub-step), (M_1 - I) x_t in the second, and the
// single-precision x+ (hi, and lo when lo_out) into shared memory.
__device__ __forceinline__ void apply_epilogue(const GroupView& g, int s, int f, const Cols& c, int r0, int j,
                                               const float (&ma)[2][4], const float (&pa)[2][4],
                                               const double2 (&x)[4], const float2 (&m1s)[4], float* hi_out,
                                               float* lo_out) {
    const int Ny = g.ny, E = g.E, VS = vec_stride(g);
    const int q = col_q(c, j), e = col_e(c, j);
    float2* M1 = (float2*)(f == 0 ? g.mx1_v : g.mx1_e);
    double2* O = (s == 2) ? (f == 0 ? g.v_t : g.e_t) : (f == 0 ? g.v_s : g.e_s);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int y = r0 + i;
        if (y >= Ny) break;
        if (!in_range(g, q, y, e) || !DNS_CK(g.status, 2 * j + 1 < VS, CK_SPEC_SMEM, y * VS + 2 * j)) continue;
        const size_t o = ((size_t)q * Ny + y) * E + e;
        const float2 m1 = (s == 2) ? m1s[i] : make_float2(ma[0][i], ma[1][i]);
        if (s == 1) M1[o] = m1;
        const double2 xn = make_double2(x[i].x + f2d(m1.x + pa[0][i]), x[i].y + f2d(m1.y + pa[1][i]));
        O[o] = xn;
        const float hx = d2f(xn.x), hy = d2f(xn.y);
        *(float2*)&hi_out[y * VS + 2 * j] = make_float2(hx, hy);
        if (lo_out)
            *(float2*)&lo_out[y * VS + 2 * j] = make_float2(d2f(xn.x - f2d(hx)), d2f(xn.y - f2d(hy)));
    }
}

// t / C for the CTA's column count C, which is EC or 2 EC (pairs with one
// mode, or both): with a compile-time EC both divisions are by constants
template <int ECC>
__device__ __forceinline__ int div_cols(int t, int C) {
    if constexpr (ECC > 0) {
        if (C == 2 * ECC) return t / (2 * ECC);
        if (C == ECC) return t / ECC;
    }
    return t / C;
}

// NYC, ECC: compile-time Ny and members per chunk of the most used group
// shapes (0: read from the group), so that the operator and vector strides of
// the products and the task divisions are constants; the arithmetic and its
// order are the same in every instantiation.
template <bool FUSE, int NYC, int ECC>
__global__ void __launch_bounds__(THREADS, 2) k_spec(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_cta(g, s, blockIdx.x, sm);
        return;
    }
    const int Ny = NYC ? NYC : g.ny, RP = NYC ? (NYC + 3) / 4 * 4 : g.rp;
    const int E = g.E, NM = g.nmodes, NKX = g.nkx;
    const int EC = ECC ? ECC : chunk_members(g), VS = 4 * EC;   // (= vec_stride(g))
    const size_t VF = (size_t)Ny * VS;                           // (= vec_floats(g))
    const int b = blockIdx.x - nrow;
    const int np1 = g.npairs - 1;                 // pair 0 is the mean mode: no CTA
    Cols c;
    c.p = 1 + b % np1;
    const int ch = b / np1;
    c.n = c.p % NKX;
    c.am = c.p / NKX;
    c.nq = c.am > 0 ? 2 : 1;
    c.q1 = (g.kz + c.am) * NKX + c.n;
    c.q2 = (g.kz - c.am) * NKX + c.n;
    c.e0 = ch * EC;
    c.ec = min(EC, E - c.e0);
    c.C = c.nq * c.ec;
    const size_t mat = (size_t)Ny * RP, slot = FUSE ? slot_floats(g) : mat;
    float* OPS = (float*)sm;                      // 4 slots: (Mv-I)^T, Pv^T, (Me-I)^T, Pe^T;
                                                  // after phase 2: D2^T, its residual in the last two
                                                  // (or, with d2fuse, D2's digit image in 0, 2, 3)
    float* D1S = OPS + 4 * slot;                  // D1^T [Ny][RP]
    float* PH = D1S + mat;                        // phi, then v+ (hi)
    float* KV = PH + VF;                          // -k^2 Nv (+ noise), then v+ (lo)
    float* GT = KV + VF;                          // G~
    float* XV = GT + VF;                          // x_t of v (single precision)
    float* XE = XV + VF;                          // x_t of eta
    float* FT = XE + VF;                          // F~
    float* EN = FT + VF;                          // eta+ (single precision)
    unsigned long long* bar = (unsigned long long*)(EN + VF);
    const unsigned bar_a = su32(bar), bar_d = su32(bar + 1), bar_m = su32(bar + 2);
    constexpr bool fuse = FUSE;                   // D2 v by the digit product below
    int* dcexp = (int*)(bar + 4);                 // fused D2 v: column exponent maxima [DCOL],
    unsigned* tslot = (unsigned*)(dcexp + DCOL);  // its TMEM base,
    int* dok = (int*)(tslot + 1);                 // its status
    const int tid = threadIdx.x;
    const bool needM = (s != 2);
    const int hidx = (s == 0) ? 0 : 1;

    if (fuse && tid < DCOL) dcexp[tid] = 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_d) : "memory");
        if (fuse) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && DNS_CK(g.status, c.p < g.npairs, CK_SPEC, c.p)) {
        const float* src = g.opsfT[hidx] + (size_t)c.p * 4 * mat;
        const unsigned mb = (unsigned)(mat * sizeof(float));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"(needM ? 5 * mb : 3 * mb) : "memory");
        bulk(D1S, g.D1T, mb, bar_a);
        if (fuse) {
            for (int k = needM ? 0 : 1; k < 4; k += needM ? 1 : 2) bulk(OPS + k * slot, src + k * mat, mb, bar_a);
        } else if (needM) {
            bulk(OPS, src, 4 * mb, bar_a);
        } else {
            bulk(OPS + mat, src + mat, mb, bar_a);
            bulk(OPS + 3 * mat, src + 3 * mat, mb, bar_a);
        }
    }

    // ---- phase 1: nonlinear terms of the pair's modes (per-plane layout) ->
    // phi, -k^2 Nv, G~ (with its RK accumulator); x_t in single precision
    {
        const size_t fs = (size_t)Ny * E * NM;
        const float2* N3 = (const float2*)g.N3;
        float2* Ae = (float2*)g.Ae;
        const int total = Ny * c.C;
        const float kx = g.kxtf[c.n];
        const bool forced = g.fn > 0 && c.n == g.fn;
        for (int i = tid; i < total; i += THREADS) {
            const int y = div_cols<ECC>(i, c.C), j = i - y * c.C;
            const int q = col_q(c, j), e = col_e(c, j);
            if (!in_range(g, q, y, e) || !DNS_CK(g.status, 2 * j + 1 < VS, CK_SPEC_SMEM, y * VS + 2 * j)) continue;
            const int mz = j < c.ec ? g.kz + c.am : g.kz - c.am;    // = q / NKX
            const float kz = g.kztf[mz];
            const size_t op = ((size_t)y * E + e) * NM + q;
            const size_t oh = ((size_t)q * Ny + y) * E + e;
            const float2 nu = N3[op], nv = N3[fs + op], nw = N3[2 * fs + op];
            float2 ae = make_float2(0.f, 0.f);
            if (s != 0) ae = Ae[oh];
            double2 xv = make_double2(0.0, 0.0), xe = xv;
            if (needM) {
                xv = g.v_t[oh];
                xe = g.e_t[oh];
            }
            const float k2 = kx * kx + kz * kz;
            const float ax = kx * nu.x + kz * nw.x, ay = kx * nu.y + kz * nw.y;   // i kx Nu + i kz Nw
            const float bx = kz * nu.x - kx * nw.x, by = kz * nu.y - kx * nw.y;   // i kz Nu - i kx Nw
            float2 kv = make_float2(-k2 * nv.x, -k2 * nv.y);
            float2 G = make_float2(-by, bx);
            if (forced && DNS_CK(g.status, mz < g.nkz, CK_SPEC, q)) {
                const size_t o = ((size_t)mz * Ny + y) * E + e, half = (size_t)g.nkz * Ny * E;
                kv.x += (float)g.noise[o].x; kv.y += (float)g.noise[o].y;
                G.x += (float)g.noise[half + o].x; G.y += (float)g.noise[half + o].y;
            }
            float2 Gt;
            if (s == 0) {
                Gt = G;
                Ae[oh] = G;
            } else if (s == 1) {
                Gt = make_float2(2.f * G.x - ae.x, 2.f * G.y - ae.y);
                Ae[oh] = make_float2((1.f / 6.f) * ae.x + (4.f / 6.f) * G.x, (1.f / 6.f) * ae.y + (4.f / 6.f) * G.y);
            } else {
                Gt = make_float2(ae.x + (1.f / 6.f) * G.x, ae.y + (1.f / 6.f) * G.y);
            }
            const int so = y * VS + 2 * j;
            *(float2*)&PH[so] = make_float2(-ay, ax);
            *(float2*)&KV[so] = kv;
            *(float2*)&GT[so] = Gt;
            if (needM) {
                *(float2*)&XV[so] = make_float2(d2f(xv.x), d2f(xv.y));
                *(float2*)&XE[so] = make_float2(d2f(xe.x), d2f(xe.y));
            }
        }
    }
    __syncthreads();
    // every thread waits for the operators (bounded); on a timeout the CTA
    // latches the status word, waits once more for the copy and leaves
    if (!__syncthreads_and(mbar_wait(bar_a, 0))) {
        if (tid == 0) {
            atomicExch(g.status, 1);
            mbar_wait(bar_a, 0);
        }
        return;
    }
    const int RB = (Ny + 3) / 4, ntask = RB * c.C;
    const size_t fs5 = (size_t)Ny * E * NM;
    float2* P5 = (float2*)g.P5;

    // ---- phase 2: F~ and (M_v - I) v_t (threads 0..127) | eta+ (threads 128..255)
    if (tid < HALF) {
        float2* Av = (float2*)g.Av;
        for (int t = tid; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, r0 = 4 * rb;
            const int q = col_q(c, j), e = col_e(c, j);
            float2 pav[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int y = r0 + i;
                pav[i] = make_float2(0.f, 0.f);
                if (s != 0 && y < Ny && in_range(g, q, y, e)) pav[i] = Av[((size_t)q * Ny + y) * E + e];
            }
            float a[2][4];
            d1mm(D1S, PH, Ny, RP, VS, r0, 2 * j, a);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int y = r0 + i;
                if (y >= Ny) break;
                if (!in_range(g, q, y, e)) continue;
                const float2 kv = *(const float2*)&KV[y * VS + 2 * j];
                const float2 F = make_float2(kv.x - a[0][i], kv.y - a[1][i]);
                const size_t oh = ((size_t)q * Ny + y) * E + e;
                float2 Ft;
                if (s == 0) {
                    Ft = F;
                    Av[oh] = F;
                } else if (s == 1) {
                    const float2 pa = pav[i];
                    Ft = make_float2(2.f * F.x - pa.x, 2.f * F.y - pa.y);
                    Av[oh] = make_float2((1.f / 6.f) * pa.x + (4.f / 6.f) * F.x, (1.f / 6.f) * pa.y + (4.f / 6.f) * F.y);
                } else {
                    const float2 pa = pav[i];
                    Ft = make_float2(pa.x + (1.f / 6.f) * F.x, pa.y + (1.f / 6.f) * F.y);
                }
                *(float2*)&FT[y * VS + 2 * j] = Ft;
            }
            // (M_v - I) x_t of the same rows and column (it needs no F~), kept in
            // the -k^2 Nv slots this thread has just read, for phase 3
            if (needM) {
                float ma[2][4];
                mm1(OPS, XV, Ny, RP, VS, r0, 2 * j, ma);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int y = r0 + i;
                    if (y >= Ny) break;
                    *(float2*)&KV[y * VS + 2 * j] = make_float2(ma[0][i], ma[1][i]);
                }
            }
        }
    } else {
        for (int t = tid - HALF; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, r0 = 4 * rb;
            double2 x[4];
            float2 m1[4];
            apply_prefetch(g, s, 1, c, r0, j, x, m1);
            float ma[2][4], pa[2][4];
            mm2(OPS + 2 * slot, OPS + 3 * slot, XE, GT, Ny, RP, VS, r0, 2 * j, needM, ma, pa);
            apply_epilogue(g, s, 1, c, r0, j, ma, pa, x, m1, EN, nullptr);
        }
    }
    __syncthreads();
    // the eta operators are no longer read: D2^T and its residual go there
    // (the generic-proxy reads of phase 2 ordered before the async-proxy writes)
    const bool d2here = !g.d2tc;     // else D2 v comes from the tensor-core digit kernel
    if (tid == 0 && d2here) {
        const unsigned mb = (unsigned)(mat * sizeof(float));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_d), "r"(2 * mb) : "memory");
        bulk(OPS + 2 * slot, g.D2T, mb, bar_d);
        bulk(OPS + 3 * slot, g.D2Tl, mb, bar_d);
    }
    // fused D2 v: the six digit slices of D2's image, two per slot, over the
    // operators phase 2 has finished with (slots 0, 2, 3), while phase 3 runs
    if (tid == 0 && fuse) {
        const unsigned b2 = (unsigned)(2 * oz::slice_a(g.kp));
        const unsigned char* img = (const unsigned char*)g.D2oz;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_d), "r"(3 * b2) : "memory");
        bulk(OPS, img, b2, bar_d);
        bulk(OPS + 2 * slot, img + b2, b2, bar_d);
        bulk(OPS + 3 * slot, img + 2 * b2, b2, bar_d);
    }

    // ---- phase 3: v+ (P_v F~, threads 0..127) | D eta and the eta planes (threads 128..255)
    if (tid < HALF) {
        for (int t = tid; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, r0 = 4 * rb;
            double2 x[4];
            float2 m1[4];
            apply_prefetch(g, s, 0, c, r0, j, x, m1);
            float ma[2][4], pa[2][4];
            mm1(OPS + slot, FT, Ny, RP, VS, r0, 2 * j, pa);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int y = r0 + i;
                float2 m = make_float2(0.f, 0.f);
                if (needM && y < Ny) m = *(const float2*)&KV[y * VS + 2 * j];
                ma[0][i] = m.x;
                ma[1][i] = m.y;
            }
            // v+ hi, lo over phi and the (M_v - I) v_t slots (each read first by
            // this thread)
            apply_epilogue(g, s, 0, c, r0, j, ma, pa, x, m1, PH, d2here ? KV : nullptr);
        }
    } else {
        for (int t = tid - HALF; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, r0 = 4 * rb;
            float a[2][4];
            d1mm(D1S, EN, Ny, RP, VS, r0, 2 * j, a);
            const int q = col_q(c, j), e = col_e(c, j);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int y = r0 + i;
                if (y >= Ny) break;
                if (!in_range(g, q, y, e)) continue;
                const size_t o = ((size_t)y * E + e) * NM + q;
                P5[3 * fs5 + o] = *(const float2*)&EN[y * VS + 2 * j];
                P5[4 * fs5 + o] = make_float2(a[0][i], a[1][i]);
            }
        }
    }
    __syncthreads();

    if (!__syncthreads_and(!d2here || mbar_wait(bar_d, 0))) {
        if (tid == 0) {
            atomicExch(g.status, 1);
            mbar_wait(bar_d, 0);
        }
        return;
    }

    // ---- fused D2 v (oz.cuh): digits of the new state's columns into slot 1,
    // the MMAs issued by one thread into TMEM; phase 4 runs under them
    const int warp = tid >> 5, lane = tid & 31;
    if (fuse) {
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                         "r"(DTCOLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        const int KP = g.kp, KC = KP / 4;
        const unsigned LBO = 128, SBO = 16 * KP;
        const size_t sb = (size_t)DCOL * KP * 2;          // bytes of one digit slice of v
        unsigned char* B = (unsigned char*)(OPS + slot);
        const double2* Vn = (s == 2) ? g.v_t : g.v_s;    // the new state (this CTA's columns written in phase 3)
        // task (complex column j, 4 consecutive k); the columns j >= C and rows
        // k >= Ny are zero
        const int j = tid % (DCOL / 2), kc = tid / (DCOL / 2);
        const bool task = kc < KC;
        double2 xv[4];
        int mr = 0, mi = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * kc + i;
            xv[i] = make_double2(0.0, 0.0);
            if (task && j < c.C && k < Ny) {
                const int q = col_q(c, j), e = col_e(c, j);
                if (in_range(g, q, k, e)) xv[i] = Vn[((size_t)q * Ny + k) * E + e];
            }
            mr = max(mr, oz::bexp(xv[i].x));
            mi = max(mi, oz::bexp(xv[i].y));
        }
        if (task) {
            atomicMax(&dcexp[2 * j], mr);
            atomicMax(&dcexp[2 * j + 1], mi);
        }
        __syncthreads();
        // (debug build) every digit of this task lands inside slot 1
        if (task && DNS_CK(g.status, (oz::NDIG - 1) * sb + (size_t)(DCOL / 8 - 1) * SBO + (size_t)(kc >> 1) * LBO + 8 * 16 <=
                                         slot * sizeof(float), CK_SPEC_SMEM, kc)) {
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const int cr = 2 * j + part;
                const int f = dcexp[cr] - 1022;           // |x| < 2^f for every x of the column
                unsigned short dg[4][oz::NDIG];
#pragma unroll
                for (int i = 0; i < 4; ++i) oz::digits(part ? xv[i].y : xv[i].x, f, dg[i]);
                const size_t off = (size_t)(cr >> 3) * SBO + (size_t)(kc >> 1) * LBO + (size_t)(cr & 7) * 16 + (kc & 1) * 8;
#pragma unroll
                for (int sd = 0; sd < oz::NDIG; ++sd) {
                    uint2 w;
                    w.x = (unsigned)dg[0][sd] | ((unsigned)dg[1][sd] << 16);
                    w.y = (unsigned)dg[2][sd] | ((unsigned)dg[3][sd] << 16);
                    *(uint2*)(B + sd * sb + off) = w;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            int good = mbar_wait(bar_d, 0) ? 1 : 0;
            if (!good) mbar_wait(bar_d, 0);                   // one more bounded wait: no copy left in flight
            if (good) {
                const unsigned tmem = *tslot;
                const unsigned idesc = oz::idesc_bf16(oz::MROWS, DCOL);
                const size_t sa = oz::slice_a(KP);
                const unsigned char* A0 = (const unsigned char*)OPS;
                const unsigned char* A2 = (const unsigned char*)(OPS + 2 * slot);
                const unsigned char* A4 = (const unsigned char*)(OPS + 3 * slot);
                const int KS = KP / 16;
                for (int L = 0; L < oz::NLEV; ++L) {
                    unsigned acc = 0;
                    for (int sd = 0; sd <= L; ++sd) {
                        const int t = L - sd;
                        const unsigned char* As = (sd < 2 ? A0 : sd < 4 ? A2 : A4) + (size_t)(sd & 1) * sa;
                        for (int ks = 0; ks < KS; ++ks) {
                            const uint64_t ad = oz::sdesc(su32(As + (size_t)ks * 2 * LBO), LBO, SBO);
                            const uint64_t bd = oz::sdesc(su32(B + t * sb + (size_t)ks * 2 * LBO), LBO, SBO);
                            oz::mma(tmem + (unsigned)(L * DCOL), ad, bd, idesc, acc);
                            acc = 1;
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_m)
                             : "memory");
            }
            *dok = good;
        }
    }

    // ---- phase 4: Dv and the compensated D2 v, 2-row x 1-complex-column tasks
    // on every thread; the v planes
    {
        const float* VH = PH;
        const float* VL = KV;
        const float* D2S = OPS + 2 * slot;
        const float* D2LS = OPS + 3 * slot;
        const int RB2 = (Ny + 1) / 2, ntask2 = RB2 * c.C;
        for (int t = tid; t < ntask2; t += THREADS) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, r0 = 2 * rb;
            float d1[2][2] = {{0.f, 0.f}, {0.f, 0.f}};    // [row][re/im]
            float sh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, sl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
            if (!d2here) {
#pragma unroll 4
                for (int k = 0; k < Ny; ++k) {
                    const float2 a1 = *(const float2*)&D1S[k * RP + r0];
                    const float2 xh = *(const float2*)&VH[k * VS + 2 * j];
                    d1[0][0] += a1.x * xh.x; d1[0][1] += a1.x * xh.y;
                    d1[1][0] += a1.y * xh.x; d1[1][1] += a1.y * xh.y;
                }
            } else
#pragma unroll 2
            for (int k = 0; k < Ny; ++k) {
                const float2 a1 = *(const float2*)&D1S[k * RP + r0];
                const float2 a2 = *(const float2*)&D2S[k * RP + r0];
                const float2 a2l = *(const float2*)&D2LS[k * RP + r0];
                const float2 xh = *(const float2*)&VH[k * VS + 2 * j];
                const float2 xl = *(const float2*)&VL[k * VS + 2 * j];
                d1[0][0] += a1.x * xh.x; d1[0][1] += a1.x * xh.y;
                d1[1][0] += a1.y * xh.x; d1[1][1] += a1.y * xh.y;
                ff_add_prod2(sh[0][0], sl[0][0], a2.x, xh.x, a2l.x, xl.x);
                ff_add_prod2(sh[0][1], sl[0][1], a2.x, xh.y, a2l.x, xl.y);
                ff_add_prod2(sh[1][0], sl[1][0], a2.y, xh.x, a2l.y, xl.x);
                ff_add_prod2(sh[1][1], sl[1][1], a2.y, xh.y, a2l.y, xl.y);
            }
            const int q = col_q(c, j), e = col_e(c, j);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int y = r0 + i;
                if (y >= Ny) break;
                if (!in_range(g, q, y, e)) continue;
                const size_t o = ((size_t)y * E + e) * NM + q;
                P5[o] = *(const float2*)&VH[y * VS + 2 * j];
                P5[fs5 + o] = make_float2(d1[i][0], d1[i][1]);
                if (d2here) P5[2 * fs5 + o] = make_float2(__fadd_rn(sh[i][0], sl[i][0]), __fadd_rn(sh[i][1], sl[i][1]));
            }
        }
    }

    // ---- fused D2 v: wait for the MMAs (bounded), rows 0..63 read back by
    // warps 0, 1, 4, 5 (TMEM lanes 32 (w & 3) .., real columns 8 (w >> 2) ..),
    // the levels combined and scaled exactly as the D2 v kernel does
    if (fuse) {
        __syncthreads();
        if (tid == 0) {
            int good = *dok;
            if (good) {
                good = mbar_wait(bar_m, 0) ? 1 : 0;
                if (!good) mbar_wait(bar_m, 0);               // do not release TMEM under running MMAs
            }
            *dok = good;
        }
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned tmem = *tslot;
        const bool ok = *dok != 0;
        if (ok && (warp & 3) < 2) {
            const int y = 32 * (warp & 3) + lane;
            const int c0 = 8 * (warp >> 2);
            float hi[8], lo[8];
            oz::combine_levels<8>(tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)c0, DCOL, hi, lo);
            if (y < Ny) {
                const float sr = oz::p2f(g.D2ozexp[y] - 14);
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const int cr = c0 + i, j = cr >> 1;
                    if (j >= c.C) break;
                    const int q = col_q(c, j), e = col_e(c, j);
                    if (!in_range(g, q, y, e)) continue;
                    // 2^(e_r + f_c) 2^-14 in two exact steps (each in the float range)
                    const float re = __fadd_rn(hi[i], lo[i]) * sr * oz::p2f(dcexp[cr] - 1022);
                    const float im = __fadd_rn(hi[i + 1], lo[i + 1]) * sr * oz::p2f(dcexp[cr + 1] - 1022);
                    P5[2 * fs5 + ((size_t)y * E + e) * NM + q] = make_float2(re, im);
                }
            }
        }
        if (!ok && tid == 0) atomicExch(g.status, 5);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(DTCOLS) : "memory");
    }
}

// ============================================================================
// The fused stage in parity blocks (k_spec_eo).  On the symmetric Chebyshev
// grid (y_j = -y_{Ny-1-j}) the per-wavenumber operators M - I and P of both
// fields commute with the reflection y -> -y (centro-symmetric) and D1
// anticommutes with it.  With every vector split into its even and odd parts,
//   x_e[i] = x[i] + x[Ny-1-i],  x_o[i] = x[i] - x[Ny-1-i]   (i < Ny / 2),
//   x_e[c] = x[c] at the centre c = (Ny-1)/2 when Ny is odd,
// a centro-symmetric operator maps even parts to even parts and odd to odd,
// and D1 maps odd to even and even to odd: each product becomes two blocks of
// half the size (NE = ceil(Ny/2) and NO = floor(Ny/2) rows), half the
// operator bytes and half the multiply-adds.  The host stores each matrix as
// its two blocks, transposed and row-padded to RP2 (eo_block_image).  Vectors
// in shared memory hold the even part in rows 0 .. NE-1 and the odd part in
// rows NE .. Ny-1; the state, forcing accumulators and outputs stay in the
// natural order in global memory, and every task converts the natural rows of
// its pair-rows (i and Ny-1-i) on the way in and out.  D2 v of the new state
// comes from the tensor-core digit kernel after the launch or (D2FF) is summed
// here in float-float, D2 and its residual in parity blocks over the eta
// operators once phase 2 is done (half the products of the natural-order
// float-float sum).
// ============================================================================

__host__ __device__ inline size_t eo_smem_bytes(const GroupView& g) {
    return (5 * eo_mat(g.ny) + 7 * vec_floats(g)) * sizeof(float) + 32;
}

template <int NYC, int ECC, int MINB, bool D2FF>
__global__ void __launch_bounds__(THREADS, MINB) k_spec_eo(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_cta(g, s, blockIdx.x, sm);
        return;
    }
    const int Ny = NYC ? NYC : g.ny;
    const int NE = (Ny + 1) / 2, NO = Ny / 2, RB2 = (NE + 1) / 2, RP2 = 2 * RB2;
    const size_t MEO = eo_mat(Ny);
    const int E = g.E, NM = g.nmodes, NKX = g.nkx;
    const int EC = ECC ? ECC : chunk_members(g), VS = 4 * EC;
    const size_t VF = (size_t)Ny * VS;
    const int b = blockIdx.x - nrow;
    const int np1 = g.npairs - 1;                 // pair 0 is the mean mode: no CTA
    Cols c;
    c.p = 1 + b % np1;
    const int ch = b / np1;
    c.n = c.p % NKX;
    c.am = c.p / NKX;
    c.nq = c.am > 0 ? 2 : 1;
    c.q1 = (g.kz + c.am) * NKX + c.n;
    c.q2 = (g.kz - c.am) * NKX + c.n;
    c.e0 = ch * EC;
    c.ec = min(EC, E - c.e0);
    c.C = c.nq * c.ec;
    float* OPS = (float*)sm;                      // 4 x MEO: (Mv-I), Pv, (Me-I), Pe in parity blocks
    float* D1S = OPS + 4 * MEO;                   // D1 in parity blocks
    float* PH = D1S + MEO;                        // phi, then v+
    float* KV = PH + VF;                          // -k^2 Nv (+ noise), then (M_v - I) v_t
    float* GT = KV + VF;                          // G~
    float* XV = GT + VF;                          // v_t (single precision)
    float* XE = XV + VF;                          // eta_t
    float* FT = XE + VF;                          // F~
    float* EN = FT + VF;                          // eta+
    unsigned long long* bar = (unsigned long long*)(EN + VF);
    const unsigned bar_a = su32(bar), bar_d = su32(bar + 1);
    const int tid = threadIdx.x;
    const bool needM = (s != 2);
    const int hidx = (s == 0) ? 0 : 1;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        if (D2FF) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_d) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && DNS_CK(g.status, c.p < g.npairs, CK_SPEC, c.p)) {
        const float* src = g.opsEO[hidx] + (size_t)c.p * 4 * MEO;
        const unsigned mb = (unsigned)(MEO * sizeof(float));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"(needM ? 5 * mb : 3 * mb) : "memory");
        bulk(D1S, g.D1EO, mb, bar_a);
        if (needM) {
            bulk(OPS, src, 4 * mb, bar_a);
        } else {
            bulk(OPS + MEO, src + MEO, mb, bar_a);
            bulk(OPS + 3 * MEO, src + 3 * MEO, mb, bar_a);
        }
    }

    // ---- phase 1: the nonlinear terms of both natural rows of each pair-row
    // -> phi, -k^2 Nv, G~ (with its RK accumulator, natural rows), x_t; their
    // even and odd parts into shared memory
    {
        const size_t fs = (size_t)Ny * E * NM;
        const float2* N3 = (const float2*)g.N3;
        float2* Ae = (float2*)g.Ae;
        const float kx = g.kxtf[c.n];
        const bool forced = g.fn > 0 && c.n == g.fn;
        const int total = NE * c.C;
        for (int i = tid; i < total; i += THREADS) {
            const int p = div_cols<ECC>(i, c.C), j = i - p * c.C;
            const int q = col_q(c, j), e = col_e(c, j);
            const int mz = j < c.ec ? g.kz + c.am : g.kz - c.am;    // = q / NKX
            const float kz = g.kztf[mz];
            const float k2 = kx * kx + kz * kz;
            const EoRows R = eo_rows(p, Ny);
            float2 ph[2], kvv[2], gt[2];
            double2 xv[2], xe[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                ph[r] = kvv[r] = gt[r] = make_float2(0.f, 0.f);
                xv[r] = xe[r] = make_double2(0.0, 0.0);
                const int y = r ? R.y1 : R.y0;
                if ((r && !R.pair) || !in_range(g, q, y, e)) continue;
                const size_t op = ((size_t)y * E + e) * NM + q;
                const size_t oh = ((size_t)q * Ny + y) * E + e;
                const float2 nu = N3[op], nv = N3[fs + op], nw = N3[2 * fs + op];
                float2 ae = make_float2(0.f, 0.f);
                if (s != 0) ae = Ae[oh];
                if (needM) {
                    xv[r] = g.v_t[oh];
                    xe[r] = g.e_t[oh];
                }
                const float ax = kx * nu.x + kz * nw.x, ay = kx * nu.y + kz * nw.y;   // i kx Nu + i kz Nw
                const float bx = kz * nu.x - kx * nw.x, by = kz * nu.y - kx * nw.y;   // i kz Nu - i kx Nw
                float2 kv = make_float2(-k2 * nv.x, -k2 * nv.y);
                float2 G = make_float2(-by, bx);
                if (forced && DNS_CK(g.status, mz < g.nkz, CK_SPEC, q)) {
                    const size_t o = ((size_t)mz * Ny + y) * E + e, half = (size_t)g.nkz * Ny * E;
                    kv.x += (float)g.noise[o].x; kv.y += (float)g.noise[o].y;
                    G.x += (float)g.noise[half + o].x; G.y += (float)g.noise[half + o].y;
                }
                float2 Gt;
                if (s == 0) {
                    Gt = G;
                    Ae[oh] = G;
                } else if (s == 1) {
                    Gt = make_float2(2.f * G.x - ae.x, 2.f * G.y - ae.y);
                    Ae[oh] = make_float2((1.f / 6.f) * ae.x + (4.f / 6.f) * G.x, (1.f / 6.f) * ae.y + (4.f / 6.f) * G.y);
                } else {
                    Gt = make_float2(ae.x + (1.f / 6.f) * G.x, ae.y + (1.f / 6.f) * G.y);
                }
                ph[r] = make_float2(-ay, ax);
                kvv[r] = kv;
                gt[r] = Gt;
            }
            if (!DNS_CK(g.status, 2 * j + 1 < VS && p < NE, CK_SPEC_SMEM, p * VS + 2 * j)) continue;
            const int se = p * VS + 2 * j, so = (NE + p) * VS + 2 * j;
            *(float2*)&PH[se] = make_float2(ph[0].x + ph[1].x, ph[0].y + ph[1].y);
            *(float2*)&KV[se] = make_float2(kvv[0].x + kvv[1].x, kvv[0].y + kvv[1].y);
            *(float2*)&GT[se] = make_float2(gt[0].x + gt[1].x, gt[0].y + gt[1].y);
            // x_t in single precision, its parts summed in single precision (the
            // increment (M - I) x_t is O(dt) x_t: one more rounding there is far below
            // the budget)
            const float2 v0 = make_float2(d2f(xv[0].x), d2f(xv[0].y)), v1 = make_float2(d2f(xv[1].x), d2f(xv[1].y));
            const float2 e0 = make_float2(d2f(xe[0].x), d2f(xe[0].y)), e1 = make_float2(d2f(xe[1].x), d2f(xe[1].y));
            if (needM) {
                *(float2*)&XV[se] = make_float2(v0.x + v1.x, v0.y + v1.y);
                *(float2*)&XE[se] = make_float2(e0.x + e1.x, e0.y + e1.y);
            }
            if (R.pair) {
                *(float2*)&PH[so] = make_float2(ph[0].x - ph[1].x, ph[0].y - ph[1].y);
                *(float2*)&KV[so] = make_float2(kvv[0].x - kvv[1].x, kvv[0].y - kvv[1].y);
                *(float2*)&GT[so] = make_float2(gt[0].x - gt[1].x, gt[0].y - gt[1].y);
                if (needM) {
                    *(float2*)&XV[so] = make_float2(v0.x - v1.x, v0.y - v1.y);
                    *(float2*)&XE[so] = make_float2(e0.x - e1.x, e0.y - e1.y);
                }
            }
        }
    }
    __syncthreads();
    // every thread waits for the operators (bounded); on a timeout the CTA
    // latches the status word, waits once more for the copy and leaves
    if (!__syncthreads_and(mbar_wait(bar_a, 0))) {
        if (tid == 0) {
            atomicExch(g.status, 1);
            mbar_wait(bar_a, 0);
        }
        return;
    }
    const int ntask = RB2 * c.C;
    const size_t fs5 = (size_t)Ny * E * NM;
    float2* P5 = (float2*)g.P5;

    // ---- phase 2: F~ and (M_v - I) v_t (threads 0..127) | eta+ (threads 128..255);
    // tasks of two pair-rows x one complex column
    if (tid < HALF) {
        float2* Av = (float2*)g.Av;
        for (int t = tid; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, p0 = 2 * rb;
            const int q = col_q(c, j), e = col_e(c, j);
            float2 pav[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                pav[r][0] = pav[r][1] = make_float2(0.f, 0.f);
                const EoRows R = eo_rows(p0 + r, Ny);
                if (s == 0 || p0 + r >= NE) continue;
                if (in_range(g, q, R.y0, e)) pav[r][0] = Av[((size_t)q * Ny + R.y0) * E + e];
                if (R.pair && in_range(g, q, R.y1, e)) pav[r][1] = Av[((size_t)q * Ny + R.y1) * E + e];
            }
            // D1 phi: the even rows contract the odd part, the odd rows the even part
            float ae[2][2], ao[2][2];
            eo2(D1S, NO, NE, RP2, PH + NE * VS, PH, VS, p0, 2 * j, ae, ao);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int p = p0 + r;
                if (p >= NE) break;
                const EoRows R = eo_rows(p, Ny);
                const float2 kve = *(const float2*)&KV[p * VS + 2 * j];
                const float2 kvo = R.pair ? *(const float2*)&KV[(NE + p) * VS + 2 * j] : make_float2(0.f, 0.f);
                const float2 Fe = make_float2(kve.x - ae[r][0], kve.y - ae[r][1]);
                const float2 Fo = make_float2(kvo.x - ao[r][0], kvo.y - ao[r][1]);
                float2 Ftn[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int y = k2 ? R.y1 : R.y0;
                    if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    // the natural row's F: half the sum or difference of its parts
                    const float2 F = !R.pair ? Fe
                                   : k2 ? make_float2(0.5f * (Fe.x - Fo.x), 0.5f * (Fe.y - Fo.y))
                                        : make_float2(0.5f * (Fe.x + Fo.x), 0.5f * (Fe.y + Fo.y));
                    const size_t oh = ((size_t)q * Ny + y) * E + e;
                    const float2 pa = pav[r][k2];
                    float2 Ft;
                    if (s == 0) {
                        Ft = F;
                        Av[oh] = F;
                    } else if (s == 1) {
                        Ft = make_float2(2.f * F.x - pa.x, 2.f * F.y - pa.y);
                        Av[oh] = make_float2((1.f / 6.f) * pa.x + (4.f / 6.f) * F.x, (1.f / 6.f) * pa.y + (4.f / 6.f) * F.y);
                    } else {
                        Ft = make_float2(pa.x + (1.f / 6.f) * F.x, pa.y + (1.f / 6.f) * F.y);
                    }
                    Ftn[k2] = Ft;
                }
                *(float2*)&FT[p * VS + 2 * j] = make_float2(Ftn[0].x + Ftn[1].x, Ftn[0].y + Ftn[1].y);
                if (R.pair)
                    *(float2*)&FT[(NE + p) * VS + 2 * j] = make_float2(Ftn[0].x - Ftn[1].x, Ftn[0].y - Ftn[1].y);
            }
            // (M_v - I) v_t of the same pair-rows and column, kept in the KV slots
            // this thread has just read, for phase 3
            if (needM) {
                float me[2][2], mo[2][2];
                eo2(OPS, NE, NO, RP2, XV, XV + NE * VS, VS, p0, 2 * j, me, mo);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int p = p0 + r;
                    if (p >= NE) break;
                    *(float2*)&KV[p * VS + 2 * j] = make_float2(me[r][0], me[r][1]);
                    if (p < NO) *(float2*)&KV[(NE + p) * VS + 2 * j] = make_float2(mo[r][0], mo[r][1]);
                }
            }
        }
    } else {
        float2* M1 = (float2*)g.mx1_e;
        double2* O = (s == 2) ? g.e_t : g.e_s;
        for (int t = tid - HALF; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, p0 = 2 * rb;
            const int q = col_q(c, j), e = col_e(c, j);
            double2 x[2][2];
            float2 m1s[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const EoRows R = eo_rows(p0 + r, Ny);
                    const int y = k2 ? R.y1 : R.y0;
                    x[r][k2] = make_double2(0.0, 0.0);
                    m1s[r][k2] = make_float2(0.f, 0.f);
                    if (p0 + r >= NE || (k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    const size_t oh = ((size_t)q * Ny + y) * E + e;
                    x[r][k2] = g.e_t[oh];
                    if (s == 2) m1s[r][k2] = M1[oh];
                }
            float mae[2][2], mao[2][2], pae[2][2], pao[2][2];
            eo2x2(OPS + 2 * MEO, OPS + 3 * MEO, NE, NO, RP2, XE, XE + NE * VS, GT, GT + NE * VS, VS, p0, 2 * j,
                  needM, mae, mao, pae, pao);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int p = p0 + r;
                if (p >= NE) break;
                const EoRows R = eo_rows(p, Ny);
                float2 hn[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int y = k2 ? R.y1 : R.y0;
                    if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    const float sg = k2 ? -1.f : 1.f;
                    const float2 ma = R.pair ? make_float2(0.5f * (mae[r][0] + sg * mao[r][0]), 0.5f * (mae[r][1] + sg * mao[r][1]))
                                             : make_float2(mae[r][0], mae[r][1]);
                    const float2 pa = R.pair ? make_float2(0.5f * (pae[r][0] + sg * pao[r][0]), 0.5f * (pae[r][1] + sg * pao[r][1]))
                                             : make_float2(pae[r][0], pae[r][1]);
                    const size_t oh = ((size_t)q * Ny + y) * E + e;
                    const float2 m1 = (s == 2) ? m1s[r][k2] : ma;
                    if (s == 1) M1[oh] = m1;
                    const double2 xn = make_double2(x[r][k2].x + f2d(m1.x + pa.x), x[r][k2].y + f2d(m1.y + pa.y));
                    O[oh] = xn;
                    hn[k2] = make_float2(d2f(xn.x), d2f(xn.y));
                    P5[3 * fs5 + ((size_t)y * E + e) * NM + q] = hn[k2];
                }
                // eta+ parts in single precision (D eta is a single-precision product)
                *(float2*)&EN[p * VS + 2 * j] = make_float2(hn[0].x + hn[1].x, hn[0].y + hn[1].y);
                if (R.pair) *(float2*)&EN[(NE + p) * VS + 2 * j] = make_float2(hn[0].x - hn[1].x, hn[0].y - hn[1].y);
            }
        }
    }
    __syncthreads();
    // D2FF: the eta operators are no longer read: D2 and its residual in parity
    // blocks go there (the generic-proxy reads of phase 2 ordered before the
    // async-proxy writes)
    if (D2FF && tid == 0) {
        const unsigned mb = (unsigned)(MEO * sizeof(float));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_d), "r"(2 * mb) : "memory");
        bulk(OPS + 2 * MEO, g.D2EO, mb, bar_d);
        bulk(OPS + 3 * MEO, g.D2lEO, mb, bar_d);
    }

    // ---- phase 3: v+ (P_v F~, threads 0..127) | D eta (threads 128..255)
    if (tid < HALF) {
        float2* M1 = (float2*)g.mx1_v;
        double2* O = (s == 2) ? g.v_t : g.v_s;
        for (int t = tid; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, p0 = 2 * rb;
            const int q = col_q(c, j), e = col_e(c, j);
            double2 x[2][2];
            float2 m1s[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const EoRows R = eo_rows(p0 + r, Ny);
                    const int y = k2 ? R.y1 : R.y0;
                    x[r][k2] = make_double2(0.0, 0.0);
                    m1s[r][k2] = make_float2(0.f, 0.f);
                    if (p0 + r >= NE || (k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    const size_t oh = ((size_t)q * Ny + y) * E + e;
                    x[r][k2] = g.v_t[oh];
                    if (s == 2) m1s[r][k2] = M1[oh];
                }
            float pe[2][2], po[2][2];
            eo2(OPS + MEO, NE, NO, RP2, FT, FT + NE * VS, VS, p0, 2 * j, pe, po);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int p = p0 + r;
                if (p >= NE) break;
                const EoRows R = eo_rows(p, Ny);
                float2 me = make_float2(0.f, 0.f), mo = me;
                if (needM) {
                    me = *(const float2*)&KV[p * VS + 2 * j];
                    if (R.pair) mo = *(const float2*)&KV[(NE + p) * VS + 2 * j];
                }
                double2 xn[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int y = k2 ? R.y1 : R.y0;
                    if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    const float sg = k2 ? -1.f : 1.f;
                    const float2 ma = R.pair ? make_float2(0.5f * (me.x + sg * mo.x), 0.5f * (me.y + sg * mo.y)) : me;
                    const float2 pa = R.pair ? make_float2(0.5f * (pe[r][0] + sg * po[r][0]), 0.5f * (pe[r][1] + sg * po[r][1]))
                                             : make_float2(pe[r][0], pe[r][1]);
                    const size_t oh = ((size_t)q * Ny + y) * E + e;
                    const float2 m1 = (s == 2) ? m1s[r][k2] : ma;
                    if (s == 1) M1[oh] = m1;
                    xn[k2] = make_double2(x[r][k2].x + f2d(m1.x + pa.x), x[r][k2].y + f2d(m1.y + pa.y));
                    O[oh] = xn[k2];
                    P5[((size_t)y * E + e) * NM + q] = make_float2(d2f(xn[k2].x), d2f(xn[k2].y));
                }
                // v+ in parity parts (over phi) for D v; with D2FF as float-float
                // pairs, the low parts over the (M_v - I) v_t slots this thread has read
                float2 he, le, ho, lo;
                eo_ff(xn[0].x, xn[1].x, he.x, le.x, ho.x, lo.x);
                eo_ff(xn[0].y, xn[1].y, he.y, le.y, ho.y, lo.y);
                *(float2*)&PH[p * VS + 2 * j] = he;
                if (R.pair) *(float2*)&PH[(NE + p) * VS + 2 * j] = ho;
                if (D2FF) {
                    *(float2*)&KV[p * VS + 2 * j] = le;
                    if (R.pair) *(float2*)&KV[(NE + p) * VS + 2 * j] = lo;
                }
            }
        }
    } else {
        for (int t = tid - HALF; t < ntask; t += HALF) {
            const int rb = div_cols<ECC>(t, c.C), j = t - rb * c.C, p0 = 2 * rb;
            const int q = col_q(c, j), e = col_e(c, j);
            float de[2][2], dq[2][2];
            eo2(D1S, NO, NE, RP2, EN + NE * VS, EN, VS, p0, 2 * j, de, dq);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int p = p0 + r;
                if (p >= NE) break;
                const EoRows R = eo_rows(p, Ny);
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    const int y = k2 ? R.y1 : R.y0;
                    if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
                    const float sg = k2 ? -1.f : 1.f;
                    const float2 d = R.pair ? make_float2(0.5f * (de[r][0] + sg * dq[r][0]), 0.5f * (de[r][1] + sg * dq[r][1]))
                                            : make_float2(de[r][0], de[r][1]);
                    P5[4 * fs5 + ((size_t)y * E + e) * NM + q] = d;
                }
            }
        }
    }
    __syncthreads();

    if (D2FF) {
        if (!__syncthreads_and(mbar_wait(bar_d, 0))) {
            if (tid == 0) {
                atomicExch(g.status, 1);
                mbar_wait(bar_d, 0);
            }
            return;
        }
    }

    // ---- phase 4: D v (and with D2FF the float-float D2 v) on every thread,
    // one pair-row x one complex column each
    for (int t = tid; t < NE * c.C; t += THREADS) {
        const int p = div_cols<ECC>(t, c.C), j = t - p * c.C;
        const int q = col_q(c, j), e = col_e(c, j);
        const EoRows R = eo_rows(p, Ny);
        float de[2], dq[2];
        eo1(D1S, NO, NE, RP2, PH + NE * VS, PH, VS, p, 2 * j, de, dq);
        float eh[2], el[2], oh[2], ol[2];
        if (D2FF) eo1ff(OPS + 2 * MEO, OPS + 3 * MEO, NE, NO, RP2, PH, KV, VS, p, 2 * j, eh, el, oh, ol);
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {
            const int y = k2 ? R.y1 : R.y0;
            if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
            const float sg = k2 ? -1.f : 1.f;
            const float2 d = R.pair ? make_float2(0.5f * (de[0] + sg * dq[0]), 0.5f * (de[1] + sg * dq[1]))
                                    : make_float2(de[0], de[1]);
            const size_t o = ((size_t)y * E + e) * NM + q;
            P5[fs5 + o] = d;
            if (D2FF) {
                const float e0 = __fadd_rn(eh[0], el[0]), e1 = __fadd_rn(eh[1], el[1]);
                const float o0 = __fadd_rn(oh[0], ol[0]), o1 = __fadd_rn(oh[1], ol[1]);
                P5[2 * fs5 + o] = R.pair ? make_float2(0.5f * (e0 + sg * o0), 0.5f * (e1 + sg * o1)) : make_float2(e0, e1);
            }
        }
    }
}

// Derivatives of a newly set state (after the upload of dns_set_state or
// dns_advance) for a group on the fused stage in parity blocks: the v and eta
// planes, D v, D eta and (D2FF) the float-float D2 v in the per-plane layout,
// computed as the fused stage computes them for the state it produces (the
// same parity parts, products and order), so a state set from outside enters
// the next sub-step as one the stage produced itself.  One CTA per (pair,
// member chunk); D2 v comes from the digit kernel where D2FF is off.
template <bool D2FF>
__global__ void __launch_bounds__(THREADS, 2) k_eo_derivs(GroupView g) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny;
    const int NE = (Ny + 1) / 2, NO = Ny / 2, RB2 = (NE + 1) / 2, RP2 = 2 * RB2;
    const size_t MEO = eo_mat(Ny);
    const int E = g.E, NM = g.nmodes, NKX = g.nkx;
    const int EC = chunk_members(g), VS = 4 * EC;
    const size_t VF = (size_t)Ny * VS;
    const int np1 = g.npairs - 1;
    Cols c;
    c.p = 1 + (int)blockIdx.x % np1;
    const int ch = (int)blockIdx.x / np1;
    c.n = c.p % NKX;
    c.am = c.p / NKX;
    c.nq = c.am > 0 ? 2 : 1;
    c.q1 = (g.kz + c.am) * NKX + c.n;
    c.q2 = (g.kz - c.am) * NKX + c.n;
    c.e0 = ch * EC;
    c.ec = min(EC, E - c.e0);
    c.C = c.nq * c.ec;
    float* D1S = (float*)sm;                      // D1, D2, its residual in parity blocks
    float* D2S = D1S + MEO;
    float* D2L = D2S + MEO;
    float* PH = D1S + (D2FF ? 3 : 1) * MEO;       // v (hi), v (lo), eta in parity parts
    float* KV = PH + VF;
    float* EN = KV + VF;
    unsigned long long* bar = (unsigned long long*)(EN + VF);
    const unsigned bar_a = su32(bar);
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned mb = (unsigned)(MEO * sizeof(float));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"((D2FF ? 3 : 1) * mb)
                     : "memory");
        bulk(D1S, g.D1EO, mb, bar_a);
        if (D2FF) {
            bulk(D2S, g.D2EO, mb, bar_a);
            bulk(D2L, g.D2lEO, mb, bar_a);
        }
    }
    const size_t fs5 = (size_t)Ny * E * NM;
    float2* P5 = (float2*)g.P5;
    for (int i = tid; i < NE * c.C; i += THREADS) {
        const int p = i / c.C, j = i - p * c.C;
        const int q = col_q(c, j), e = col_e(c, j);
        const EoRows R = eo_rows(p, Ny);
        double2 v[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)}, et[2] = {v[0], v[1]};
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {
            const int y = k2 ? R.y1 : R.y0;
            if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
            const size_t oh = ((size_t)q * Ny + y) * E + e, o = ((size_t)y * E + e) * NM + q;
            v[k2] = g.v_t[oh];
            et[k2] = g.e_t[oh];
            P5[o] = make_float2(d2f(v[k2].x), d2f(v[k2].y));
            P5[3 * fs5 + o] = make_float2(d2f(et[k2].x), d2f(et[k2].y));
        }
        if (!DNS_CK(g.status, 2 * j + 1 < VS && p < NE, CK_SPEC_SMEM, p * VS + 2 * j)) continue;
        float2 he, le, ho, lo;
        eo_ff(v[0].x, v[1].x, he.x, le.x, ho.x, lo.x);
        eo_ff(v[0].y, v[1].y, he.y, le.y, ho.y, lo.y);
        const float2 h0 = make_float2(d2f(et[0].x), d2f(et[0].y)), h1 = make_float2(d2f(et[1].x), d2f(et[1].y));
        *(float2*)&PH[p * VS + 2 * j] = he;
        *(float2*)&KV[p * VS + 2 * j] = le;
        *(float2*)&EN[p * VS + 2 * j] = make_float2(h0.x + h1.x, h0.y + h1.y);
        if (R.pair) {
            *(float2*)&PH[(NE + p) * VS + 2 * j] = ho;
            *(float2*)&KV[(NE + p) * VS + 2 * j] = lo;
            *(float2*)&EN[(NE + p) * VS + 2 * j] = make_float2(h0.x - h1.x, h0.y - h1.y);
        }
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(bar_a, 0))) {
        if (tid == 0) {
            atomicExch(g.status, 1);
            mbar_wait(bar_a, 0);
        }
        return;
    }
    for (int t = tid; t < NE * c.C; t += THREADS) {
        const int p = t / c.C, j = t - p * c.C;
        const int q = col_q(c, j), e = col_e(c, j);
        const EoRows R = eo_rows(p, Ny);
        float de[2], dq[2], fe[2], fq[2];
        eo1(D1S, NO, NE, RP2, PH + NE * VS, PH, VS, p, 2 * j, de, dq);
        eo1(D1S, NO, NE, RP2, EN + NE * VS, EN, VS, p, 2 * j, fe, fq);
        float eh[2], el[2], oh[2], ol[2];
        if (D2FF) eo1ff(D2S, D2L, NE, NO, RP2, PH, KV, VS, p, 2 * j, eh, el, oh, ol);
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2) {
            const int y = k2 ? R.y1 : R.y0;
            if ((k2 && !R.pair) || !in_range(g, q, y, e)) continue;
            const float sg = k2 ? -1.f : 1.f;
            const size_t o = ((size_t)y * E + e) * NM + q;
            P5[fs5 + o] = R.pair ? make_float2(0.5f * (de[0] + sg * dq[0]), 0.5f * (de[1] + sg * dq[1]))
                                 : make_float2(de[0], de[1]);
            P5[4 * fs5 + o] = R.pair ? make_float2(0.5f * (fe[0] + sg * fq[0]), 0.5f * (fe[1] + sg * fq[1]))
                                     : make_float2(fe[0], fe[1]);
            if (D2FF) {
                const float e0 = __fadd_rn(eh[0], el[0]), e1 = __fadd_rn(eh[1], el[1]);
                const float o0 = __fadd_rn(oh[0], ol[0]), o1 = __fadd_rn(oh[1], ol[1]);
                P5[2 * fs5 + o] = R.pair ? make_float2(0.5f * (e0 + sg * o0), 0.5f * (e1 + sg * o1)) : make_float2(e0, e1);
            }
        }
    }
}

}  // namespace spc

bool spec_supported(const GroupView& g) {
    return !g.lin && g.npairs > 1 && spc::smem_bytes(g) + 1024 <= 227 * 1024;
}

// The fused D2 v for a group whose stage runs with d2fuse set (callers set it
// before asking): the digit image exists (d2tc), the CTA's columns fit the MMA's
// N, and every slice with the rows that follow it lies inside shared memory.
bool spec_d2fuse_supported(const GroupView& g) {
    return g.d2fuse && g.d2tc && !g.lin && g.ny <= 64 && g.kp % 16 == 0 && 4 * spc::chunk_members(g) <= spc::DCOL &&
           spc::fused_d2_fits(g) && spec_supported(g);
}

size_t spec_smem_bytes(const GroupView& g) {
    const size_t b = g.spec_eo ? spc::eo_smem_bytes(g) : spc::smem_bytes(g), m = mean_smem_bytes(g);
    return b > m ? b : m;
}

// (D2 v from the digit kernel after the launch, or with spec_eoff summed inside)
bool spec_eo_supported(const GroupView& g) {
    return !g.lin && g.npairs > 1 && (g.d2tc || g.spec_eoff) && !g.d2fuse && spc::eo_smem_bytes(g) + 1024 <= 227 * 1024;
}

size_t spec_eo_mat_floats(int ny) { return spc::eo_mat(ny); }

static size_t eo_derivs_smem_bytes(const GroupView& g) {
    return ((g.spec_eoff ? 3 : 1) * spc::eo_mat(g.ny) + 3 * spc::vec_floats(g)) * sizeof(float) + 32;
}

void launch_eo_derivs(const GroupView& g, cudaStream_t st) {
    const int ctas = (g.npairs - 1) * spc::chunks(g);
    if (g.spec_eoff) spc::k_eo_derivs<true><<<ctas, spc::THREADS, eo_derivs_smem_bytes(g), st>>>(g);
    else spc::k_eo_derivs<false><<<ctas, spc::THREADS, eo_derivs_smem_bytes(g), st>>>(g);
}

// The parity blocks of a matrix A (Ny x Ny, row-major), R(j) = Ny-1-j, NO =
// Ny/2, the centre c = NO when Ny is odd.  Centro-symmetric A (A[R i][R j] =
// A[i][j]): even block Ae[i][k] = A[i][k] + A[i][R k] (k < NO), 2 A[i][c]
// (k = c), with the centre row A[c][k], A[c][c]; odd block Ao[i][k] = A[i][k] -
// A[i][R k].  Anti-centro-symmetric A (A[R i][R j] = -A[i][j], D1): even rows
// from the odd part, Aeo[i][k] = A[i][k] - A[i][R k] (centre row A[c][k]); odd
// rows from the even part, Aoe[i][k] = A[i][k] + A[i][R k], 2 A[i][c] (k = c).
// Each block transposed [k][row], rows padded to RP2: the even output rows'
// block first (KE inputs), then the odd output rows' block.
void spec_eo_image(const double* A, int ny, bool anti, float* out, bool residual) {
    const int NE = spc::eo_ne(ny), NO = ny / 2, RP2 = spc::eo_rp(ny);
    const size_t mat = spc::eo_mat(ny);
    for (size_t i = 0; i < mat; ++i) out[i] = 0.f;
    auto a = [&](int i, int j) { return A[(size_t)i * ny + j]; };
    const int KE = anti ? NO : NE, KO = anti ? NE : NO;
    float* be = out;
    float* bo = out + (size_t)KE * RP2;
    for (int i = 0; i < NE; ++i)
        for (int k = 0; k < KE; ++k) {
            double v;
            if (i < NO) v = (!anti && k == NO) ? 2.0 * a(i, NO) : (anti ? a(i, k) - a(i, ny - 1 - k) : a(i, k) + a(i, ny - 1 - k));
            else v = a(NO, k);                    // the centre row (odd Ny)
            be[(size_t)k * RP2 + i] = residual ? (float)(v - (double)(float)v) : (float)v;
        }
    for (int i = 0; i < NO; ++i)
        for (int k = 0; k < KO; ++k) {
            double v;
            if (anti) v = (k == NO) ? 2.0 * a(i, NO) : a(i, k) + a(i, ny - 1 - k);
            else v = a(i, k) - a(i, ny - 1 - k);
            bo[(size_t)k * RP2 + i] = residual ? (float)(v - (double)(float)v) : (float)v;
        }
}

// the shapes with their own instantiation: (Ny, members per chunk)
#define DNS_SPEC_SHAPES(X) X(63, 4) X(63, 2) X(63, 8)

void launch_spec(const GroupView& g, int s, cudaStream_t st) {
    const int ctas = mean_row_ctas(g) + (g.npairs - 1) * spc::chunks(g);
    const size_t sm = spec_smem_bytes(g);
    if (g.spec_eo) {
        const int ec = spc::chunk_members(g);
        const bool three = g.spec_minb == 3, ff = g.spec_eoff != 0;
#define DNS_GO(a, b, m)                                                                      \
        {                                                                                    \
            if (ff) spc::k_spec_eo<a, b, m, true><<<ctas, spc::THREADS, sm, st>>>(g, s);     \
            else spc::k_spec_eo<a, b, m, false><<<ctas, spc::THREADS, sm, st>>>(g, s);       \
        }
#define DNS_CASE(a, b)                                                                       \
        if (g.ny == a && ec == b) {                                                          \
            if (three) DNS_GO(a, b, 3) else DNS_GO(a, b, 2)                                  \
            return;                                                                          \
        }
        DNS_SPEC_SHAPES(DNS_CASE)
#undef DNS_CASE
        if (three) DNS_GO(0, 0, 3) else DNS_GO(0, 0, 2)
#undef DNS_GO
        return;
    }
    if (g.d2fuse) {
        spc::k_spec<true, 0, 0><<<ctas, spc::THREADS, sm, st>>>(g, s);
        return;
    }
    const int ec = spc::chunk_members(g);
#define DNS_CASE(a, b)                                                      \
    if (g.ny == a && ec == b) {                                             \
        spc::k_spec<false, a, b><<<ctas, spc::THREADS, sm, st>>>(g, s);     \
        return;                                                             \
    }
    DNS_SPEC_SHAPES(DNS_CASE)
#undef DNS_CASE
    spc::k_spec<false, 0, 0><<<ctas, spc::THREADS, sm, st>>>(g, s);
}

void set_attributes_spec() {
    allow_max_dynamic_smem(spc::k_spec<false, 0, 0>);
    allow_max_dynamic_smem(spc::k_spec<true, 0, 0>);
#define DNS_EO(a, b)                                        \
    allow_max_dynamic_smem(spc::k_spec_eo<a, b, 2, false>);  \
    allow_max_dynamic_smem(spc::k_spec_eo<a, b, 3, false>);  \
    allow_max_dynamic_smem(spc::k_spec_eo<a, b, 2, true>);   \
    allow_max_dynamic_smem(spc::k_spec_eo<a, b, 3, true>);
#define DNS_CASE(a, b) allow_max_dynamic_smem(spc::k_spec<false, a, b>); DNS_EO(a, b)
    DNS_SPEC_SHAPES(DNS_CASE)
#undef DNS_CASE
    DNS_EO(0, 0)
#undef DNS_EO
    allow_max_dynamic_smem(spc::k_eo_derivs<false>);
    allow_max_dynamic_smem(spc::k_eo_derivs<true>);
}

}  // namespace dnsk
