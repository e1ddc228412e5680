// D2 v of the mixed path on tensor cores, accurate to the last bit of single
// precision although D2's rows cancel (Sec. 3.1 y-derivatives; the collocation
// D2 has entries up to ~N^4 / 10 whose products with v sum to a far smaller
// result, so any sum accumulated in FP32 loses ~1e-5 of |D2 v|).
//
// Error-free splitting into integer digits (the splitting of Ozaki et al.,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication", 2012, with small integers in place of floating
// slices): every row r of D2 is scaled by a power of two 2^e_r above its
// largest entry and written as S = 6 signed 7-bit digits, D2_rk = 2^e_r
// sum_s a_s 2^(-7(s+1)); every real column c of v (one mode, member, real or
// imaginary part) likewise with 2^f_c.  Digits are integers of magnitude
// <= 127, exact in BF16, their products exact, and a level L = s + t sums at
// most 6 x 64 products of at most 127^2: below 2^24, so the FP32 accumulators
// of tcgen05 (kind::f16, BF16 operands) hold every level EXACTLY.  The levels
// L <= 5 are kept (the rest and the digits beyond the sixth weigh < 2^-42 of
// the row and column scales: about 3e-9 of |D2 v| at My = 65 and 97), combined
// in float-float and scaled back:
//   D2 v = 2^(e_r + f_c) sum_L 2^(-7(L+2)) acc_L.
// One CTA per 16 complex columns (32 real columns, 6 accumulators of 32 TMEM
// columns each; two CTAs per SM; four warps read the accumulators back); M = 128 with the 64 used rows (Ny <= 64), rows 64..127 reading
// the shared memory that follows and never read back.  The digit image of D2
// arrives by one TMA bulk copy; v is read from the FP64 state and split by the
// CTA.  Every mbarrier wait is bounded; on a timeout the CTA latches the status
// word, waits once more for what it issued, releases its TMEM and leaves.
#include "dns_internal.hpp"
#include "ff.cuh"
#include "oz.cuh"
#include <cstdint>
#include <cstring>
#include <vector>

namespace dnsk {

namespace oz {

constexpr int THREADS = 256;
constexpr int CC = 16;             // complex columns per CTA
constexpr int NCOL = 2 * CC;       // real columns = TMEM columns per level

__host__ __device__ inline size_t slice_b(int KP) { return (size_t)NCOL * KP * 2; }
__host__ __device__ inline size_t smem_total(int KP) {
    return NDIG * slice_a(KP) + NDIG * slice_b(KP) + NCOL * sizeof(int) + 32;
}

__global__ void __launch_bounds__(THREADS, 2) k_d2v_tc(GroupView g, const double2* __restrict__ V) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int Ny = g.ny, KP = g.kp, E = g.E, NM = g.nmodes;
    const int ncc = NM * E;                       // complex columns of the group (H order: q major)
    const int cc0 = blockIdx.x * CC;
    const size_t sa = slice_a(KP), sb = slice_b(KP);
    unsigned char* A = sm;                        // [NDIG][64 rows x KP]
    unsigned char* B = sm + NDIG * sa;            // [NDIG][NCOL x KP]
    int* cexp = (int*)(B + NDIG * sb);            // [NCOL] biased exponent maxima
    unsigned* tslot = (unsigned*)(cexp + NCOL);
    unsigned long long* bars = (unsigned long long*)(tslot + 4);
    const unsigned bar_a = su32(&bars[0]), bar_m = su32(&bars[1]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned LBO = 128, SBO = 16 * KP;
    constexpr unsigned TCOLS = 256;               // NLEV * NCOL = 192, allocated as 256

    if (tid < NCOL) cexp[tid] = 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        // one arrival per issuing lane (one lane per level, below)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_m), "r"(NLEV) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned bytes = (unsigned)(NDIG * sa);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(su32(A)), "l"(g.D2oz), "r"(bytes), "r"(bar_a) : "memory");
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;

    // ---- B: tasks (complex column j, 4 consecutive k); pass 1 the column
    // exponents, pass 2 the digits (each thread keeps its values in registers)
    const int KC = KP / 4, ntask = CC * KC;
    constexpr int TPT = 1;                        // tasks per thread: CC * KC <= THREADS (KP <= 64)
    double2 xv[TPT][4];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        const int t = tid + u * THREADS;
        const int j = t % CC, kc = t / CC;
        const int cc = cc0 + j;
        const bool col = t < ntask && cc < ncc;
        const int q = col ? cc / E : 0, e = col ? cc - q * E : 0;
        int mr = 0, mi = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = kc * 4 + i;
            double2 x = make_double2(0.0, 0.0);
            if (col && k < Ny && DNS_CK(g.status, q < NM && e < E, CK_D2V, cc)) x = V[((size_t)q * Ny + k) * E + e];
            xv[u][i] = x;
            mr = max(mr, bexp(x.x));
            mi = max(mi, bexp(x.y));
        }
        if (t < ntask) {
            atomicMax(&cexp[2 * j], mr);
            atomicMax(&cexp[2 * j + 1], mi);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        const int t = tid + u * THREADS;
        if (t >= ntask) break;
        const int j = t % CC, kc = t / CC;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int c = 2 * j + part;
            const int f = cexp[c] - 1022;         // |x| < 2^f for every x of the column
            unsigned short dg[4][NDIG];
#pragma unroll
            for (int i = 0; i < 4; ++i) digits(part ? xv[u][i].y : xv[u][i].x, f, dg[i]);
            // k = 4 kc .. 4 kc + 3: half of a core-matrix row (8 k, 16 bytes)
            const size_t off = (size_t)(c >> 3) * SBO + (size_t)(kc >> 1) * LBO + (size_t)(c & 7) * 16 + (kc & 1) * 8;
#pragma unroll
            for (int s = 0; s < NDIG; ++s) {
                uint2 w;
                w.x = (unsigned)dg[0][s] | ((unsigned)dg[1][s] << 16);
                w.y = (unsigned)dg[2][s] | ((unsigned)dg[3][s] << 16);
                *(uint2*)(B + s * sb + off) = w;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- the MMAs: level L into TMEM columns [L NCOL, (L + 1) NCOL), issued by
    // lane L of warp 0 (tcgen05.mma has single-thread semantics: each lane
    // issues its own sequence; a level's MMAs stay in one lane, in order, and
    // each lane's commit arrives once on bar_m)
    __shared__ int ok_flag;
    if (warp == 0) {
        int mine = 1;
        if (lane < NLEV) mine = mbar_wait(bar_a, 0) ? 1 : 0;
        int good = __all_sync(0xffffffffu, mine);
        if (!good && lane == 0) mbar_wait(bar_a, 0);   // one more bounded wait: no copy left in flight
        if (good && lane < NLEV) {
            const unsigned idesc = idesc_bf16(MROWS, NCOL);
            const int KS = KP / 16, L = lane;
            unsigned acc = 0;
            for (int s = 0; s <= L; ++s) {
                const int t = L - s;
                for (int ks = 0; ks < KS; ++ks) {
                    const uint64_t ad = sdesc(su32(A + s * sa + (size_t)ks * 2 * LBO), LBO, SBO);
                    const uint64_t bd = sdesc(su32(B + t * sb + (size_t)ks * 2 * LBO), LBO, SBO);
                    mma(tmem + (unsigned)(L * NCOL), ad, bd, idesc, acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_m)
                         : "memory");
        }
        __syncwarp();
        if (lane == 0) {
            if (good) {
                good = mbar_wait(bar_m, 0) ? 1 : 0;
                if (!good) mbar_wait(bar_m, 0);       // do not release TMEM under running MMAs
            }
            ok_flag = good;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = ok_flag != 0;

    // ---- epilogue: rows 0..63; warp w (0, 1, 4, 5) reads TMEM lanes 32 (w & 3)
    // (the lanes its sub-partition may access) and real columns 16 (w >> 2) ..
    if (ok && (warp & 3) < 2) {
        const int y = 32 * (warp & 3) + lane;
        const unsigned trow = tmem + ((unsigned)(32 * (warp & 3)) << 16);
        const int er = y < Ny ? g.D2ozexp[y] : 0;
        const size_t fs = (size_t)Ny * E * NM;
        float2* P5 = (float2*)g.P5;
        const int c0 = 16 * (warp >> 2);
        float hi[16], lo[16];
        combine_levels<16>(trow + (unsigned)c0, NCOL, hi, lo);
        if (y < Ny) {
            const float sr = p2f(er - 14);
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const int c = c0 + i, j = c >> 1, cc = cc0 + j;
                if (cc >= ncc) break;
                const int q = cc / E, e = cc - q * E;
                if (!DNS_CK(g.status, q < NM && e < E && y < Ny, CK_D2V, cc)) continue;
                // 2^(e_r + f_c) 2^-14 in two exact steps (each in the float range)
                const float re = __fadd_rn(hi[i], lo[i]) * sr * p2f(cexp[c] - 1022);
                const float im = __fadd_rn(hi[i + 1], lo[i + 1]) * sr * p2f(cexp[c + 1] - 1022);
                P5[2 * fs + ((size_t)y * E + e) * NM + q] = make_float2(re, im);
            }
        }
    }
    if (!ok && tid == 0) atomicExch(g.status, 5);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

}  // namespace oz

bool d2v_tc_supported(const GroupView& g) { return g.ny <= 64 && !g.lin; }

size_t d2v_tc_smem_bytes(const GroupView& g) { return oz::smem_total(g.kp); }

size_t d2v_tc_image_bytes(const GroupView& g) { return oz::NDIG * oz::slice_a(g.kp); }

void launch_d2v_tc(const GroupView& g, const double2* v, cudaStream_t st) {
    const int ctas = (g.nmodes * g.E + oz::CC - 1) / oz::CC;
    oz::k_d2v_tc<<<ctas, oz::THREADS, d2v_tc_smem_bytes(g), st>>>(g, v);
}

void set_attributes_d2v_tc() { allow_max_dynamic_smem(oz::k_d2v_tc); }

// Host image of D2's digits: per interior row r the exponent e_r with
// max_k |D2_rk| < 2^e_r, and NDIG slices of 7-bit signed digits of
// D2_rk 2^-e_r (rounded to 49 fraction bits), each slice 64 rows x KP in the
// no-swizzle K-major core-matrix layout; rows >= Ny and k >= Ny are zero.
static inline uint16_t bf16_of_small_int(int d) {
    const float f = (float)(d < 0 ? -d : d);
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)((u >> 16) | (d < 0 ? 0x8000u : 0u));
}

void d2v_tc_image(const std::vector<double>& D2i, int ny, int kp, std::vector<uint16_t>& img, std::vector<int>& rexp) {
    const size_t slice = (size_t)64 * kp;                 // bf16 elements
    img.assign(oz::NDIG * slice, 0);
    rexp.assign(64, 0);
    const size_t sbo = (size_t)8 * kp;                    // elements between 8-row groups
    for (int r = 0; r < ny; ++r) {
        double mx = 0.0;
        for (int k = 0; k < ny; ++k) mx = std::max(mx, std::fabs(D2i[(size_t)r * ny + k]));
        int e = 0;
        if (mx > 0.0) {
            std::frexp(mx, &e);                           // mx = m 2^e, 0.5 <= m < 1: mx < 2^e
        }
        rexp[r] = e;
        for (int k = 0; k < ny; ++k) {
            const double x = std::ldexp(D2i[(size_t)r * ny + k], -e);   // |x| < 1, exact
            const double ax = std::fabs(x);
            uint64_t X = (uint64_t)std::llround(std::ldexp(ax, oz::FBITS));
            if (X >= (1ull << oz::FBITS)) X = (1ull << oz::FBITS) - 1;
            for (int s = 0; s < oz::NDIG; ++s) {
                const int u = (int)((X >> (7 * (oz::NDIG - 1 - s))) & 127u);
                const size_t off = (size_t)(r >> 3) * sbo + (size_t)(k >> 3) * 64 + (size_t)(r & 7) * 8 + (k & 7);
                img[s * slice + off] = u ? bf16_of_small_int(x < 0 ? -u : u) : 0;
            }
        }
    }
}

}  // namespace dnsk
