// Tensor-core implicit apply of the mixed path (Eqs. CN1, CN2 in increment
// form, Sec. 3.2): per wavenumber pair (n, |m|) and field (v or eta),
//   x+ = x_t + ((M_h - I) x_t + P_h F~)
// with the pair's operators [M_h - I | P_h] (Ny x 2Ny) applied to the stacked
// right-hand side [x_t ; F~] of all members and both modes +-m, as one tcgen05
// GEMM with K = 2 KP (KP = Ny padded to 16).  Every operand is split into three
// BF16 pieces (the operators on the host from their FP64 values, x_t and F~ in
// the kernel from single precision) and the six significant piece products are
// accumulated in FP32 in TMEM; the increment is then added to the FP64 state
// with one double add per element.
//   Sub-step 1 (h = 1/2): one accumulator, K over [x_t ; F~].
//   Sub-step 2 (h = 1):   (M_1 - I) x_t and P_1 F~ in two accumulators; the first
//                         is also stored (single precision) for sub-step 3.
//   Sub-step 3 (h = 1):   P_1 F~ only, plus the stored (M_1 - I) x_t.
// The MMA runs with M = 128: rows 0..63 are the operator rows (Ny <= 64), rows
// 64..127 read whatever follows in shared memory and their results are never
// read.  The pair's operator image (3 pieces, 64 rows) arrives by one TMA bulk
// copy; columns beyond 128 are done in passes.  Every
// mbarrier wait is bounded; on a timeout the CTA latches the status word,
// waits once more for what it issued, releases its TMEM and leaves.
#include "dns_internal.hpp"
#include "mbar.cuh"
#include "cvt.cuh"
#include "mean.cuh"
#include <cuda_bf16.h>
#include <cstring>
#include <vector>

namespace dnsk {

namespace htc {

constexpr int THREADS = 256;
constexpr int MROWS = 128;     // MMA rows (64 used)
constexpr int NPMAX = 128;     // columns per pass

// Shared-memory matrix descriptor, no swizzle, K-major core matrices (8 rows x
// 16 bytes): LBO = distance between core matrices along K, SBO = between
// 8-row groups.
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D F32, A = B = BF16, K-major.
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

// Split x into three BF16 pieces, x = h + m + l exactly: each piece keeps the
// leading 8 significand bits of what is left (truncation, by masking the low
// 16 bits), and each remainder is exact in float.  Integer masks and FP32
// subtractions only: the float -> BF16 conversion instructions would issue to
// the slow conversion pipe.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    const unsigned ux = __float_as_uint(x) & 0xFFFF0000u;
    const float r1 = x - __uint_as_float(ux);
    const unsigned u1 = __float_as_uint(r1) & 0xFFFF0000u;
    const float r2 = r1 - __uint_as_float(u1);
    const unsigned u2 = __float_as_uint(r2) & 0xFFFF0000u;
    h = __ushort_as_bfloat16((unsigned short)(ux >> 16));
    m = __ushort_as_bfloat16((unsigned short)(u1 >> 16));
    l = __ushort_as_bfloat16((unsigned short)(u2 >> 16));
}

// Column geometry of a pair: N = 2 nq E real columns (mode, member, re/im), in
// passes of NP (a multiple of 32, at most 128).
struct Geo {
    int N, NP, passes;
};
__host__ __device__ inline Geo geo_of(int nq, int E) {
    Geo g;
    g.N = 2 * nq * E;
    const int n32 = (g.N + 31) / 32 * 32;
    g.NP = n32 < NPMAX ? n32 : NPMAX;
    g.passes = (g.N + g.NP - 1) / g.NP;
    return g;
}

// shared memory: A [3][64 rows][2 KP] | B [3][NPMAX or less][2 KP] (reused as the
// staging of the increments [2][64][NP + 1] floats) | tmem slot | 2 mbarriers
__host__ __device__ inline size_t piece_a(int KP) { return (size_t)64 * 2 * KP * 2; }
__host__ __device__ inline size_t bytes_a(int KP) { return 3 * piece_a(KP); }
__host__ __device__ inline size_t bytes_b(int KP, int NP) {
    const size_t b = (size_t)3 * NP * 2 * KP * 2;
    const size_t st = (size_t)2 * 64 * (NP + 1) * 4;
    const size_t tail = piece_a(KP);      // rows 64..127 of the last A piece read this far
    size_t m = b > st ? b : st;
    return m > tail ? m : tail;
}
__host__ __device__ inline size_t smem_total(int KP, int NP) { return bytes_a(KP) + bytes_b(KP, NP) + 64; }

__global__ void __launch_bounds__(THREADS, 1) k_helm_tc(GroupView g, int s) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int E = g.E;
    const int Ny = g.ny, KP = g.kp, NKX = g.nkx;
    // leading CTAs: rows of the mean-flow update (see the SIMT kernel)
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_rows(g, s, blockIdx.x % E, (blockIdx.x / E) * (THREADS / 32), sm);
        return;
    }
    const int b = blockIdx.x - nrow;
    const int p = b % g.npairs, f = b / g.npairs;
    const int n = p % NKX, am = p / NKX;
    if (!g.lin && n == 0 && am == 0) return;   // the mean mode (DNS groups)
    const int hi = (s == 0) ? 0 : 1;
    const int nq = am > 0 ? 2 : 1;
    const int q1 = (g.kz + am) * NKX + n, q2 = (g.kz - am) * NKX + n;
    const Geo G = geo_of(nq, E);
    const int K2 = 2 * KP;
    unsigned char* A = sm;
    unsigned char* B = sm + bytes_a(KP);
    unsigned* tslot = (unsigned*)(B + bytes_b(KP, G.NP));
    unsigned long long* bars = (unsigned long long*)(B + bytes_b(KP, G.NP) + 16);
    const unsigned bar_a = su32(&bars[0]), bar_m = su32(&bars[1]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned LBO = 128, SBO = 16 * K2;           // bytes; same for A and B
    const size_t pieceA = piece_a(KP), pieceB = (size_t)G.NP * K2 * 2;
    unsigned ncols = 32;
    while (ncols < 2u * (unsigned)G.NP) ncols <<= 1;

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)bytes_a(KP);
        const unsigned char* src = (const unsigned char*)g.Htc[hi] + ((size_t)p * 2 + f) * bytes_a(KP);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(su32(A)), "l"(src), "r"(bytes), "r"(bar_a) : "memory");
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;

    const double* X = (const double*)(f == 0 ? g.v_t : g.e_t);
    const float* F = (const float*)(f == 0 ? g.Fv : g.Fe);
    float* M1 = (float*)(f == 0 ? g.mx1_v : g.mx1_e);
    double* O = (double*)((s == 2) ? (f == 0 ? g.v_t : g.e_t) : (f == 0 ? g.v_s : g.e_s));
    const int twoE = 2 * E;
    __shared__ int ok_flag;
    bool ok = true;
    for (int pass = 0; pass < G.passes && ok; ++pass) {
        const int cbase = pass * G.NP;
        const int ncur = (G.N - cbase) < G.NP ? (G.N - cbase) : G.NP;
        // ---- B = [x_t ; F~] (columns: mode, member, re/im), 8 consecutive k per task
        const int KC = K2 / 8;
        const int kc0 = (s == 2) ? KP / 8 : 0;        // sub-step 3 needs the F~ half only
        const int ntask = G.NP * (KC - kc0);
        // each thread's tasks (up to TPT of 8 consecutive k for one column): all
        // global loads first, then the splits and shared stores
        constexpr int TPT = 2;
        for (int i0 = threadIdx.x; i0 < ntask; i0 += THREADS * TPT) {
            float xs[TPT][8];
#pragma unroll
            for (int u = 0; u < TPT; ++u) {
                const int i = i0 + u * THREADS;
                const int nl = i % G.NP, kc = kc0 + i / G.NP;
                const int cg = cbase + nl;
                const bool col = i < ntask && nl < ncur;
                const int which = col ? cg / twoE : 0, r = col ? cg - which * twoE : 0;
                const int q = which == 0 ? q1 : q2;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int k = kc * 8 + t;
                    const bool xpart = k < KP;
                    const int y = xpart ? k : k - KP;
                    float x = 0.f;
                    if (col && y < Ny) {
                        const size_t o = ((size_t)q * Ny + y) * twoE + r;
                        x = xpart ? d2f(X[o]) : F[o];
                    }
                    xs[u][t] = x;
                }
            }
#pragma unroll
            for (int u = 0; u < TPT; ++u) {
                const int i = i0 + u * THREADS;
                if (i >= ntask) break;
                const int nl = i % G.NP, kc = kc0 + i / G.NP;
                __nv_bfloat16 hv[8], mv[8], lv[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) split3(xs[u][t], hv[t], mv[t], lv[t]);
                const size_t off = (size_t)(nl >> 3) * SBO + (size_t)kc * LBO + (size_t)(nl & 7) * 16;
                *(uint4*)(B + off) = *(const uint4*)hv;
                *(uint4*)(B + pieceB + off) = *(const uint4*)mv;
                *(uint4*)(B + 2 * pieceB + off) = *(const uint4*)lv;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) {
            int good = 1;
            if (pass == 0) {
                good = mbar_wait(bar_a, 0) ? 1 : 0;
                if (!good) mbar_wait(bar_a, 0);           // one more bounded wait: no copy left in flight
            }
            if (good) {
                const unsigned idesc = idesc_bf16(MROWS, G.NP);
                const int pa[6] = {2, 0, 1, 1, 0, 0}, pb[6] = {0, 2, 1, 0, 1, 0};
                auto run = [&](unsigned dcol, int ks0, int ks1) {
                    unsigned acc = 0;
                    for (int ks = ks0; ks < ks1; ++ks)
                        for (int t = 0; t < 6; ++t) {
                            const uint64_t ad = sdesc(su32(A + pa[t] * pieceA + (size_t)ks * 2 * LBO), LBO, SBO);
                            const uint64_t bd = sdesc(su32(B + pb[t] * pieceB + (size_t)ks * 2 * LBO), LBO, SBO);
                            mma(tmem + dcol, ad, bd, idesc, acc);
                            acc = 1;
                        }
                };
                const int KS = K2 / 16, KH = KP / 16;
                if (s == 0) {
                    run(0, 0, KS);
                } else if (s == 1) {
                    run(0, 0, KH);
                    run((unsigned)G.NP, KH, KS);
                } else {
                    run((unsigned)G.NP, KH, KS);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(bar_m) : "memory");
                // thread 0 waits for the MMAs; the barrier below hands the result
                // (and the completed accumulators) to every thread
                good = mbar_wait(bar_m, (unsigned)(pass & 1)) ? 1 : 0;
                if (!good) mbar_wait(bar_m, (unsigned)(pass & 1));   // do not touch B or TMEM under running MMAs
            }
            ok_flag = good;
        }
        __syncthreads();
        ok = ok_flag != 0;                // uniform across the CTA
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue 1: TMEM rows 0..63 (warps 0, 1, 4, 5) -> staging [2][64][NP+1]
        float* stD = (float*)B;
        float* stM = stD + 64 * (G.NP + 1);
        if (ok && (warp & 3) < 2) {
            const int y = 32 * (warp & 3) + lane;
            const unsigned trow = tmem + ((unsigned)(32 * (warp & 3)) << 16);
            const int c0 = (warp >> 2) * (G.NP / 2);
            for (int c = c0; c < c0 + G.NP / 2; c += 16) {
                float a[16], bb[16];
                if (s == 0) {
                    ld16(trow + c, a);
#pragma unroll
                    for (int t = 0; t < 16; ++t) stD[y * (G.NP + 1) + c + t] = a[t];
                } else if (s == 1) {
                    ld16(trow + c, a);
                    ld16(trow + G.NP + c, bb);
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        stM[y * (G.NP + 1) + c + t] = a[t];
                        stD[y * (G.NP + 1) + c + t] = a[t] + bb[t];
                    }
                } else {
                    ld16(trow + G.NP + c, bb);
#pragma unroll
                    for (int t = 0; t < 16; ++t) stD[y * (G.NP + 1) + c + t] = bb[t];
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // ---- epilogue 2: coalesced state update in the per-mode layout.  Each
        // thread loads its UNR elements before storing any (in sub-step 3 the
        // output overwrites x_t, which would otherwise serialise the loads).
        if (ok) {
            constexpr int UNR = 8;
            const int total = Ny * ncur;
            for (int i0 = threadIdx.x; i0 < total; i0 += THREADS * UNR) {
                double xv[UNR];
                float dv[UNR], mv[UNR];
                size_t ov[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int i = i0 + u * THREADS;
                    ov[u] = 0;
                    if (i < total) {
                        const int y = i / ncur, nl = i - y * ncur;
                        const int cg = cbase + nl;
                        const int which = cg / twoE, r = cg - which * twoE;
                        const int q = which == 0 ? q1 : q2;
                        ov[u] = ((size_t)q * Ny + y) * twoE + r;
                        xv[u] = X[ov[u]];
                        dv[u] = stD[y * (G.NP + 1) + nl];
                        if (s == 2) dv[u] += M1[ov[u]];
                        mv[u] = stM[y * (G.NP + 1) + nl];
                    }
                }
                // stores only after every load of the batch (no global store
                // between the loads: they may alias, which would serialise them)
#pragma unroll
                for (int u = 0; u < UNR; ++u)
                    if (i0 + u * THREADS < total) {
                        if (s == 1) M1[ov[u]] = mv[u];
                        O[ov[u]] = xv[u] + f2d(dv[u]);
                    }
            }
        }
        __syncthreads();          // staging and B are rewritten by the next pass
    }
    if (!ok && threadIdx.x == 0) atomicExch(g.status, 4);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace htc

bool helm_tc_supported(const GroupView& g) { return g.ny <= 64 && g.E <= 64; }

size_t helm_tc_smem_bytes(const GroupView& g) {
    const htc::Geo G = htc::geo_of(2, g.E);
    size_t b = htc::smem_total(g.kp, G.NP);
    const size_t m = mean_smem_bytes(g);
    return b > m ? b : m;
}

void launch_helm_tc(const GroupView& g, int s, cudaStream_t st) {
    htc::k_helm_tc<<<mean_row_ctas(g) + 2 * g.npairs, htc::THREADS, helm_tc_smem_bytes(g), st>>>(g, s);
}

void set_attributes_helm_tc() { allow_max_dynamic_smem(htc::k_helm_tc); }

// Host images of [M - I | P] per (pair, field) for one sub-step length: three
// BF16 pieces of the FP64 operators, 64 rows x 2 KP (zero padded), in the
// no-swizzle K-major core-matrix layout of the kernel's A descriptors.
// ops: [npairs][4][Ny][Ny] (Mv, Pv, Me, Pe).  Output [npairs][2 fields][3][...].
static inline uint16_t bf16_bits_h(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}
static inline float bf16_val_h(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

std::vector<uint16_t> helm_tc_a_images(const std::vector<double>& ops, int npairs, int ny, int kp) {
    const int K2 = 2 * kp;
    const size_t piece = (size_t)64 * K2;                  // bf16 elements
    const size_t img = 3 * piece;
    const size_t sbo = 16 * (size_t)K2 / 2;                // elements between 8-row groups
    const size_t nn = (size_t)ny * ny;
    std::vector<uint16_t> out((size_t)npairs * 2 * img, 0);
    for (int p = 0; p < npairs; ++p)
        for (int f = 0; f < 2; ++f) {
            const double* Mo = &ops[((size_t)p * 4 + 2 * f) * nn];
            const double* Po = &ops[((size_t)p * 4 + 2 * f + 1) * nn];
            uint16_t* dst = &out[((size_t)p * 2 + f) * img];
            for (int m = 0; m < ny; ++m)
                for (int k = 0; k < K2; ++k) {
                    double x = 0.0;
                    if (k < kp) {
                        if (k < ny) x = Mo[(size_t)m * ny + k] - (m == k ? 1.0 : 0.0);
                    } else if (k - kp < ny) {
                        x = Po[(size_t)m * ny + (k - kp)];
                    }
                    const uint16_t h = bf16_bits_h((float)x);
                    const double r1 = x - (double)bf16_val_h(h);
                    const uint16_t mm = bf16_bits_h((float)r1);
                    const double r2 = r1 - (double)bf16_val_h(mm);
                    const uint16_t l = bf16_bits_h((float)r2);
                    const size_t off = (size_t)(m >> 3) * sbo + (size_t)(k >> 3) * 64 + (size_t)(m & 7) * 8 + (k & 7);
                    dst[off] = h;
                    dst[piece + off] = mm;
                    dst[2 * piece + off] = l;
                }
        }
    return out;
}

}  // namespace dnsk
