// Tensor-core y-contraction of the mixed path (Sec. 3.1: y-derivatives by
// one shared Chebyshev matrix applied to every mode and member):
//   [Dv ; D2v] = [D1_int ; D2_int] v,   D eta = D1_int eta
// as one tcgen05 GEMM per 256-column tile, D (TMEM, FP32) = A (128 x K) B^T
// with A = [D1_int ; D2_int] (rows 0..63 and 64..127, zero padded) and B the
// tile's columns (128 real columns of v, 128 of eta; K = interior y padded to
// 16).  Near-FP32 accuracy from BF16 tensor cores by splitting every operand
// in three BF16 pieces, x = x_h + x_m + x_l, and accumulating the six products
// that matter (l h, h l, m m, m h, h m, h h) into the same TMEM accumulator.
//
// Data movement: the three A pieces arrive by TMA bulk copy (prepared on the
// host in the no-swizzle K-major core-matrix layout); B is read from the FP64
// state, split, and written to shared memory in the same layout; the epilogue
// reads TMEM with tcgen05.ld, stages through shared memory and writes the
// per-plane layout with coalesced stores.  Every mbarrier wait is bounded; on
// a timeout the kernel latches the status word, still releases its TMEM, and
// leaves.
#include "dns_internal.hpp"
#include "mbar.cuh"
#include "mean.cuh"
#include <cuda_bf16.h>
#include <cstring>
#include <vector>

namespace dnsk {

namespace tc {

constexpr int THREADS = 256;          // 8 warps; warp w reads TMEM lanes 32 (w % 4) in the epilogue
// Tile width NCOL (template parameter, 128 or 64): real columns = TMEM columns,
// half of v, half of eta; NCOL / 4 complex columns per field.  The narrow tile
// doubles the CTAs where the wide one would leave most SMs idle.
constexpr int MROWS = 128;

// Shared-memory matrix descriptor, no swizzle, K-major core matrices
// (8 rows x 16 bytes each, rows 16 bytes apart): LBO = distance between core
// matrices along K, SBO = distance between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    return d;                           // base offset 0, layout 0 (no swizzle)
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
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

struct Tile {
    int QT, EBT;
};

template <int NCOL>
__host__ __device__ inline Tile tile_of(int E) {
    constexpr int JT = NCOL / 4;
    Tile t;
    t.EBT = E < JT ? E : JT;
    t.QT = JT / t.EBT;
    return t;
}

// Shared memory: A pieces [3][128 x KP] bf16 | B pieces [3][NCOL x KP] bf16 (reused
// as the output staging [3][64][JT+1] float2) | tmem slot | 2 mbarriers.
// staging row stride JT + 1 (odd: conflict-free column writes)
__host__ __device__ inline size_t smem_a(int KP) { return (size_t)3 * MROWS * KP * 2; }
template <int NCOL>
__host__ __device__ inline size_t smem_b(int KP) {
    size_t b = (size_t)3 * NCOL * KP * 2;
    size_t st = (size_t)3 * 64 * (NCOL / 4 + 1) * 8;
    return b > st ? b : st;
}
template <int NCOL>
__host__ __device__ inline size_t smem_total(int KP) { return smem_a(KP) + smem_b<NCOL>(KP) + 64; }

template <int NCOL>
__global__ void __launch_bounds__(THREADS, 2) k_yderiv_tc(GroupView g, const double2* __restrict__ V,
                                                          const double2* __restrict__ H, int sprev) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int SROW = NCOL / 4 + 1;
    const int Ny = g.ny, KP = g.kp, E = g.E, NM = g.nmodes;
    const Tile T = tile_of<NCOL>(E);
    if (mean_finish_rows(g, sprev, (E + T.EBT - 1) / T.EBT, sm)) return;
    const int q0 = blockIdx.x * T.QT, e0 = blockIdx.y * T.EBT;
    unsigned char* A = sm;
    unsigned char* B = sm + smem_a(KP);
    unsigned* tslot = (unsigned*)(B + smem_b<NCOL>(KP));
    unsigned long long* bars = (unsigned long long*)(B + smem_b<NCOL>(KP) + 16);
    const unsigned bar_a = su32(&bars[0]), bar_m = su32(&bars[1]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned LBO = 128, SBO = 16 * KP;            // bytes
    const size_t pieceA = (size_t)MROWS * KP * 2, pieceB = (size_t)NCOL * KP * 2;

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(3 * pieceA);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(su32(A)), "l"(g.Atc), "r"(bytes), "r"(bar_a) : "memory");
    }
    // B: column n = f*(NCOL/2) + 2 j + c, j = qq*EBT + el (H order), rows k (interior y)
    // each thread's tasks (8 consecutive k of one column): all global loads
    // first, then the splits and the shared stores
    const int KC = KP / 8;
    constexpr int TPT = 4;
    const FastDiv dEBT((unsigned)T.EBT), dQT((unsigned)T.QT);
    for (int i0 = threadIdx.x; i0 < NCOL * KC; i0 += THREADS * TPT) {
        float xs[TPT][8];
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int i = i0 + u * THREADS;
            const int n = i % NCOL, kc = i / NCOL;
            const int f = n / (NCOL / 2), r = n % (NCOL / 2), j = r >> 1, c = r & 1;
            const int qq = (int)dEBT.div((unsigned)j), el = j - qq * T.EBT;
            const int q = q0 + qq, e = e0 + el;
            const bool ok = i < NCOL * KC && (qq < T.QT) && (q < NM) && (e < E);
            const double* src = (const double*)(f == 0 ? V : H);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = kc * 8 + t;
                float x = 0.f;
                if (ok && k < Ny) x = (float)src[(((size_t)q * Ny + k) * E + e) * 2 + c];
                xs[u][t] = x;
            }
        }
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int i = i0 + u * THREADS;
            if (i >= NCOL * KC) break;
            const int n = i % NCOL, kc = i / NCOL;
            __nv_bfloat16 hv[8], mv[8], lv[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) split3(xs[u][t], hv[t], mv[t], lv[t]);
            const size_t off = (size_t)(n >> 3) * SBO + (size_t)kc * LBO + (size_t)(n & 7) * 16;
            *(uint4*)(B + off) = *(const uint4*)hv;
            *(uint4*)(B + pieceB + off) = *(const uint4*)mv;
            *(uint4*)(B + 2 * pieceB + off) = *(const uint4*)lv;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    __shared__ int ok_flag;
    if (threadIdx.x == 0) {
        int ok = mbar_wait(bar_a, 0) ? 1 : 0;
        if (!ok) mbar_wait(bar_a, 0);          // one more bounded wait: no copy left in flight
        if (ok) {
            const unsigned idesc = idesc_bf16(MROWS, NCOL);
            // piece pairs (a, b) by increasing magnitude: l h, h l, m m, m h, h m, h h
            const int pa[6] = {2, 0, 1, 1, 0, 0}, pb[6] = {0, 2, 1, 0, 1, 0};
            unsigned acc = 0;
            for (int ks = 0; ks < KP / 16; ++ks)
                for (int t = 0; t < 6; ++t) {
                    const uint64_t ad = sdesc(su32(A + pa[t] * pieceA + (size_t)ks * 2 * LBO), LBO, SBO);
                    const uint64_t bd = sdesc(su32(B + pb[t] * pieceB + (size_t)ks * 2 * LBO), LBO, SBO);
                    mma(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_m)
                         : "memory");
        }
        ok_flag = ok;
    }
    __syncthreads();
    bool ok = ok_flag != 0;
    if (ok) {
        ok = mbar_wait(bar_m, 0);
        if (!ok) mbar_wait(bar_m, 0);          // do not release TMEM under running MMAs
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4).. (output rows m) and the
        // column half w / 4 (v or eta)
        float2* stage = (float2*)B;    // [3][64][SROW]: Dv, D2v, D eta
        const int m = 32 * (warp & 3) + lane;
        const int f = warp >> 2;
        const unsigned trow = tmem + ((unsigned)(32 * (warp & 3)) << 16);
        int fld;
        if (m < 64) fld = (f == 0) ? 0 : 2;
        else fld = (f == 0) ? 1 : -1;
        if (fld >= 0) {
            const int y = m & 63;
            for (int c0 = f * (NCOL / 2); c0 < (f + 1) * (NCOL / 2); c0 += 16) {
                float v[16];
                ld16(trow + c0, v);
                const int j0 = (c0 % (NCOL / 2)) >> 1;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    stage[((size_t)fld * 64 + y) * SROW + j0 + t] = make_float2(v[2 * t], v[2 * t + 1]);
            }
        }
    } else {
        atomicExch(g.status, 3);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
    if (!ok) return;
    // coalesced writes in the per-plane layout P[field][(y E + e) NM + q]
    const float2* stage = (const float2*)B;
    float2* P = (float2*)g.P5;
    const size_t fs = (size_t)Ny * E * NM;
    const int per = T.EBT * T.QT;
    const FastDiv dNP((unsigned)(Ny * per)), dPER((unsigned)per);
    for (int i = threadIdx.x; i < 3 * Ny * per; i += THREADS) {
        const int fld = (int)dNP.div((unsigned)i), r = i - fld * (Ny * per);
        const int y = (int)dPER.div((unsigned)r), r2 = r - y * per;
        const int el = (int)dQT.div((unsigned)r2), qq = r2 - el * T.QT;
        const int q = q0 + qq, e = e0 + el;
        if (q >= NM || e >= E) continue;
        const int dst_field = fld == 0 ? 1 : (fld == 1 ? 2 : 4);
        P[dst_field * fs + ((size_t)y * E + e) * NM + q] = stage[((size_t)fld * 64 + y) * SROW + qq * T.EBT + el];
    }
    // the fields themselves (rounded to float) in the same layout; each thread
    // loads its UNR elements before storing any
    constexpr int UNR = 4;
    for (int i0 = threadIdx.x; i0 < Ny * per; i0 += THREADS * UNR) {
        double2 a[UNR], b[UNR];
        size_t o[UNR];
        bool in[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int i = i0 + u * THREADS;
            const int y = (int)dPER.div((unsigned)i), r2 = i - y * per;
            const int el = (int)dQT.div((unsigned)r2), qq = r2 - el * T.QT;
            const int q = q0 + qq, e = e0 + el;
            in[u] = i < Ny * per && q < NM && e < E;
            o[u] = ((size_t)y * E + e) * NM + q;
            if (in[u]) {
                const size_t h = ((size_t)q * Ny + y) * E + e;
                a[u] = V[h];
                b[u] = H[h];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (in[u]) {
                P[o[u]] = make_float2((float)a[u].x, (float)a[u].y);
                P[3 * fs + o[u]] = make_float2((float)b[u].x, (float)b[u].y);
            }
    }
}

}  // namespace tc

bool yderiv_tc_supported(const GroupView& g) { return g.ny <= 64 && g.E <= 64; }

// the narrow tile where the wide one, with the group's concurrent member
// blocks, gives fewer than two CTAs per SM (with enough concurrent blocks the
// finer grid only adds per-CTA overhead)
static int yderiv_tc_width(const GroupView& g) {
    const tc::Tile t = tc::tile_of<128>(g.E);
    const long ctas = (long)((g.nmodes + t.QT - 1) / t.QT) * ((g.E + t.EBT - 1) / t.EBT);
    return ctas * (g.nblk > 0 ? g.nblk : 1) < 2 * 152 ? 64 : 128;
}

size_t yderiv_tc_smem_bytes(const GroupView& g) {
    return yderiv_tc_width(g) == 64 ? tc::smem_total<64>(g.kp) : tc::smem_total<128>(g.kp);
}

template <int NCOL>
static void launch_yderiv_tc_w(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev) {
    const tc::Tile t = tc::tile_of<NCOL>(g.E);
    dim3 grid((g.nmodes + t.QT - 1) / t.QT, (g.E + t.EBT - 1) / t.EBT);
    grid.y += mean_finish_extra_rows(g, grid.x, sprev);
    tc::k_yderiv_tc<NCOL><<<grid, tc::THREADS, tc::smem_total<NCOL>(g.kp), st>>>(g, v, e, sprev);
}

void launch_yderiv_tc(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev) {
    if (yderiv_tc_width(g) == 64) launch_yderiv_tc_w<64>(g, v, e, st, sprev);
    else launch_yderiv_tc_w<128>(g, v, e, st, sprev);
}

void set_attributes_yderiv_tc() {
    allow_max_dynamic_smem(tc::k_yderiv_tc<64>);
    allow_max_dynamic_smem(tc::k_yderiv_tc<128>);
}

// Host image of A = [D1_int ; D2_int] split into three BF16 pieces, in the
// no-swizzle K-major core-matrix layout the kernel's descriptors describe.
static inline uint16_t bf16_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;                     // round to nearest even
    return (uint16_t)(u >> 16);
}
static inline float bf16_val(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

std::vector<uint16_t> yderiv_tc_a_image(const std::vector<double>& D1i, const std::vector<double>& D2i, int ny, int kp) {
    const size_t piece = (size_t)tc::MROWS * kp;
    std::vector<uint16_t> img(3 * piece, 0);
    const size_t sbo = 16 * (size_t)kp / 2;   // in bf16 elements (16 kp bytes)
    for (int m = 0; m < tc::MROWS; ++m) {
        const int y = m & 63;
        const std::vector<double>& D = m < 64 ? D1i : D2i;
        for (int k = 0; k < kp; ++k) {
            double x = (y < ny && k < ny) ? D[(size_t)y * ny + k] : 0.0;
            uint16_t h = bf16_bits((float)x);
            double r1 = x - (double)bf16_val(h);
            uint16_t mm = bf16_bits((float)r1);
            double r2 = r1 - (double)bf16_val(mm);
            uint16_t l = bf16_bits((float)r2);
            const size_t off = (size_t)(m >> 3) * sbo + (size_t)(k >> 3) * 64 + (size_t)(m & 7) * 8 + (k & 7);
            img[off] = h;
            img[piece + off] = mm;
            img[2 * piece + off] = l;
        }
    }
    return img;
}

}  // namespace dnsk
