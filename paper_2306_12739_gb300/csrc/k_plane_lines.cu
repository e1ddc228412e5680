// Single-precision physical-space stage (mixed path), one CTA per (interior
// y-plane, member), organised around line ownership.  Same mathematics as the
// other plane kernels (paper Sec. 3.1-3.2): u, w from v, eta; 12 inverse
// transforms with 2/3-rule zero padding; N_i = u d_x u_i + v d_y u_i + w d_z u_i;
// plane means <uv>, <wv>; 3 forward transforms with truncation.
//
// Every 1-D transform of length N = N1 x N2 belongs to one group of
// G = max(N1, N2) threads inside one warp: N2 tasks of N1-point DFTs in
// registers, twiddle, an exchange through the group's own shared slot under
// __syncwarp, N1 tasks of N2-point DFTs.  A CTA-wide barrier is needed only
// where data crosses lines, which gives four phases:
//   1  z transforms of the nine fields that need one (u_i, d_y u_i, d_z u_i)
//      into kept-column storage COL[f][z][n], n <= Kx;
//   2a x transforms of u, v, w into physical planes;
//   2b per line pair (rows p and p + Mz/2, packed as one complex line) and
//      component i: x transforms of d_x u_i (the columns of u_i times i kx),
//      d_y u_i and d_z u_i, the products summed in registers of the threads
//      that hold the same points, and the forward x transform of N_i started
//      straight from those registers; the kept kx of N_i overwrite the two rows
//      of u_i's columns, which only this group reads;
//   3  forward z transforms of the kept columns, truncation, output.
// Row strides, slot strides and a row permutation inside blocks of eight z
// rows are chosen so that a warp's shared accesses fall in distinct banks.
// Rotational form (ROT): N = omega x u instead of u . grad u; phase 1 then
// transforms u, v, w and the three vorticity components (6 fields), and each
// phase-2b group inverts the two vorticity lines its component needs.
#include "dns_internal.hpp"
#include "dft.cuh"
#include "ff.cuh"
#include <type_traits>


namespace dnsk {

namespace pln {

using namespace dft;
typedef float2 C;

__device__ __forceinline__ C f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ C conjf2(C a) { return make_float2(a.x, -a.y); }

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E> struct SFor {
    template <typename F> __device__ __forceinline__ static void run(F& f) {
        f(std::integral_constant<int, B>());
        SFor<B + 1, E>::run(f);
    }
};
template <int E> struct SFor<E, E> {
    template <typename F> __device__ __forceinline__ static void run(F&) {}
};

// asynchronous global -> shared copies (completion awaited with cp_async_wait)
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }
// smallest v >= a with v % m == r
constexpr int pad_to(int a, int m, int r) { return a + ((r - a % m) % m + m) % m; }
constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t al16(size_t a) { return (a + 15) / 16 * 16; }

// Column row stride (complex words), z-row permutation on/off and physical
// row stride (floats) per plane size: the conflict-free choices for the access
// patterns below (lanes = t * units-per-warp + group).
constexpr int col_stride(int mx, int mz) {
    return mx == 16 ? 6 : mx == 32 ? 12 : mx == 48 ? 18 : (mz == 16 ? 24 : 22);
}
constexpr int col_perm(int mx, int mz) {
    return (mx == 16 && mz > 16) || mx == 48 || (mx == 64 && mz > 16) ? 1 : 0;
}
constexpr int pln_stride(int mx, int mz) {
    return mz == 16 ? (mx == 16 ? 24 : mx == 64 ? 20 : 18)
         : mz == 32 ? (mx == 16 ? 40 : 36)
         : mz == 48 ? (mx == 16 ? 56 : mx == 64 ? 52 : 50)
         : (mx == 16 ? 72 : 68);
}

template <int MX, int MZ, bool ROT = false>
struct LCfg {
    static constexpr int KX = (MX - 1) / 3, KZ = (MZ - 1) / 3;
    static constexpr int NKX = KX + 1, NKZ = 2 * KZ + 1, NM = NKX * NKZ;
    static constexpr int X1 = Split<MX>::N1, X2 = Split<MX>::N2;
    static constexpr int Z1 = Split<MZ>::N1, Z2 = Split<MZ>::N2;
    static constexpr int GX = cmax(X1, X2), GZ = cmax(Z1, Z2);   // threads per line
    static constexpr int UX = 32 / GX, UZ = 32 / GZ;              // lines per warp
    static constexpr int HP = MZ / 2;                             // line pairs
    static constexpr int NF1 = ROT ? 6 : 9;                       // fields with a z stage
    static constexpr int NU1 = NF1 * NKX, NU2 = 3 * HP, NU3 = 3 * NKX;
    static constexpr int NT0 = cmax(NU2 * GX, (NU1 + 1) / 2 * GZ);
    static constexpr int NT = rup(NT0, 32) > 1024 ? 1024 : rup(NT0, 32);
    static constexpr int NW = NT / 32;
    static constexpr int NSX = NT / GX, NSZ = NT / GZ;            // lines in flight
    static constexpr int S = col_stride(MX, MZ);
    static constexpr int PERM = col_perm(MX, MZ);
    static constexpr int MZP = pln_stride(MX, MZ);
    static constexpr int CFS = MZ * S;
    static constexpr int NKXB = pad_to(NKX, 16, UZ == 4 ? 12 : 8);   // staged input row stride
    static constexpr int ZR = Z2 + 1, XR = X2 + 1, XRF = X1 + 1;     // exchange row strides
    static constexpr int RSZ = pad_to(Z1 * ZR, 16, UZ == 4 ? 12 : 6);
    static constexpr int RSX = pad_to(cmax(cmax(X1 * XR, X2 * XRF), MX), 16, UX == 4 ? 12 : 6);
    static constexpr int PLANE = MX * MZ;
    static constexpr size_t B_COL = 0;
    static constexpr size_t B_PLN = al16(B_COL + sizeof(C) * NF1 * CFS);
    static constexpr size_t PLN_BYTES = smax(sizeof(float) * 3 * MX * MZP, sizeof(C) * 5 * NKZ * NKXB);
    static constexpr size_t B_X = al16(B_PLN + PLN_BYTES);
    static constexpr size_t B_TW = al16(B_X + sizeof(C) * smax((size_t)NSX * RSX, (size_t)NSZ * RSZ));
    static constexpr size_t B_K = B_TW + sizeof(C) * (MX + MZ);
    static constexpr size_t B_RED = al16(B_K + sizeof(float) * (NKX + NKZ + NKZ * NKXB));
    static constexpr size_t BYTES = B_RED + (2 + 2 * 32) * sizeof(double);
    static constexpr int MINB = (2 * (BYTES + 1024) <= 228 * 1024 && NT * 2 * 64 <= 65536) ? 2 : 1;
    static_assert(MZ % 8 == 0, "z-row permutation works in blocks of eight");
    static_assert(X2 - 1 <= KX && Z2 - 1 <= KZ, "first DFT slot lies in the kept band");
};

template <int MX, int MZ>
__device__ __forceinline__ int zrow(int z) {
    if (!LCfg<MX, MZ>::PERM) return z;
    const int b = z & 7;
    return (z & ~7) | ((2 * b) & 7) | (b >> 2);
}

template <int MX, int MZ, bool ROT>
__global__ void __launch_bounds__(LCfg<MX, MZ, ROT>::NT, LCfg<MX, MZ, ROT>::MINB)
k_plane_lines(GroupView g, const double* __restrict__ Ucur, const double* __restrict__ Wcur) {
    typedef LCfg<MX, MZ, ROT> K;
    constexpr int KX = K::KX, KZ = K::KZ, NKX = K::NKX, NKZ = K::NKZ, NM = K::NM;
    constexpr int X1 = K::X1, X2 = K::X2, Z1 = K::Z1, Z2 = K::Z2, HP = K::HP;
    constexpr int GX = K::GX, UX = K::UX, UZ = K::UZ, NT = K::NT;
    constexpr int S = K::S, CFS = K::CFS, MZP = K::MZP, NKXB = K::NKXB;
    constexpr int ZR = K::ZR, XR = K::XR, XRF = K::XRF, RSZ = K::RSZ, RSX = K::RSX;
    constexpr int FSB = NKZ * NKXB;   // staged input field stride
    extern __shared__ __align__(16) unsigned char smem[];
    C* COL = (C*)(smem + K::B_COL);
    float* PLN = (float*)(smem + K::B_PLN);
    C* BASE = (C*)(smem + K::B_PLN);     // staged inputs, phase 1 only (shares PLN's space)
    C* XCH = (C*)(smem + K::B_X);
    C* twx = (C*)(smem + K::B_TW);
    C* twz = twx + MX;
    float* kxs = (float*)(smem + K::B_K);
    float* kzs = kxs + NKX;
    float* k2s = kzs + NKZ;
    double* red = (double*)(smem + K::B_RED);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y = blockIdx.x, e = blockIdx.y, E = g.E, Ny = g.ny, My = g.my;
    const size_t fs = (size_t)Ny * E * NM;
    const size_t off0 = ((size_t)y * E + e) * NM;
    // the grid covers the interior planes and members exactly; the kept-mode
    // count is the compile-time one (checked by the debug build)
    if (!DNS_CK(g.status, y < Ny && e < E && NM == g.nmodes, CK_PLANE_LINES, (long long)y * E + e)) return;

    // ---- stage inputs [f][m][n] (padded rows) and tables, all copies in flight at once
    {
        const C* P = (const C*)g.P5;
        for (int i = tid; i < 5 * NM; i += NT) {
            const int f = i / NM, q = i - f * NM, mi = q / NKX, n = q - mi * NKX;
            cp_async8(BASE + f * FSB + mi * NKXB + n, P + f * fs + off0 + q);
        }
        for (int i = tid; i < MX; i += NT) cp_async8(twx + i, g.twxf + i);
        for (int i = tid; i < MZ; i += NT) cp_async8(twz + i, g.twzf + i);
        for (int i = tid; i < NKX; i += NT) cp_async4(kxs + i, g.kxtf + i);
        for (int i = tid; i < NKZ; i += NT) cp_async4(kzs + i, g.kztf + i);
        for (int q = tid; q < NM; q += NT) {
            const int mi = q / NKX;
            cp_async4(k2s + mi * NKXB + q - mi * NKX, g.k2invf + q);
        }
    }
    const float Um = (float)Ucur[(size_t)e * My + y + 1];
    const float Wm = (float)Wcur[(size_t)e * My + y + 1];
    mean_dy_row(g.D1, Ucur + (size_t)e * My, Wcur + (size_t)e * My, My, y + 1, red);
    cp_async_wait();
    __syncthreads();
    const float dUm = (float)red[0];
    const float dWm = (float)red[1];

    // spectral value at mode (mi, n) of u_comp (kind 0), d_y u_comp (kind 1)
    // or d_z u_comp (kind 2); u, w from v, eta as u = i (kx Dv - kz eta) / k^2,
    // w = i (kz Dv + kx eta) / k^2 (d_y: D2v, D eta in place of Dv, eta), the
    // (0, 0) mode from the mean flow.  Loads and selects only, no divergence
    // on the mode.
    auto gen = [&](int kind, int comp, int mi, int n) -> C {
        const C* B = BASE + mi * NKXB + n;
        const float kz = kzs[mi];
        C r;
        if (comp == 1) {
            r = kind == 1 ? B[FSB] : B[0];
        } else {
            const float kx = kxs[n], ki = k2s[mi * NKXB + n];
            const C a = kind == 1 ? B[2 * FSB] : B[FSB];
            const C b = kind == 1 ? B[4 * FSB] : B[3 * FSB];
            float ax, ay;
            if (comp == 0) { ax = (kx * a.x - kz * b.x) * ki; ay = (kx * a.y - kz * b.y) * ki; }
            else { ax = (kz * a.x + kx * b.x) * ki; ay = (kz * a.y + kx * b.y) * ki; }
            r = f2(-ay, ax);
            const float mv = kind == 1 ? (comp == 0 ? dUm : dWm) : (comp == 0 ? Um : Wm);
            if (mi == KZ && n == 0) r = f2(mv, 0.f);
        }
        if (kind == 2) r = f2(-kz * r.y, kz * r.x);
        return r;
    };

    // ---- phase 1: z transforms, line (f, n), f = 3 kind + comp
    {
        const int t = lane / UZ, gi = lane % UZ;
        C* X = XCH + (warp * UZ + gi) * RSZ;
        for (int u0 = warp * UZ; u0 < K::NU1; u0 += K::NSZ) {
            const int u = u0 + gi;
            const bool act = u < K::NU1;
            const int f = act ? u / NKX : 0, n = act ? u - f * NKX : 0;
            const int kind = f / 3, comp = f - 3 * kind;
            // rotational form: f = 3 + c is omega_c (x: dw/dy - dv/dz, y: eta, z: dv/dx - du/dy)
            auto field = [&](int mi) -> C {
                if (!ROT || f < 3) return gen(kind, comp, mi, n);
                if (comp == 1) return BASE[3 * FSB + mi * NKXB + n];
                if (comp == 0) {
                    const C a = gen(1, 2, mi, n), b = gen(2, 1, mi, n);
                    return f2(a.x - b.x, a.y - b.y);
                }
                const C vv = BASE[mi * NKXB + n], b = gen(1, 0, mi, n);
                const float kx = kxs[n];
                return f2(-kx * vv.y - b.x, kx * vv.x - b.y);
            };
            if (act && t < Z2) {
                C v[Z1];
                // slot n1 holds z = Z2 n1 + t: blocks of slots wholly inside the
                // kept band or the padding are resolved at compile time
                auto ld = [&](auto ic) {
                    constexpr int n1 = decltype(ic)::value, z0 = Z2 * n1, z1 = z0 + Z2 - 1;
                    constexpr bool lo = z1 <= KZ, hi = z0 >= MZ - KZ, pad = z0 > KZ && z1 < MZ - KZ;
                    if constexpr (pad) {
                        v[n1] = f2(0.f, 0.f);
                    } else {
                        const int z = z0 + t;
                        const bool in_lo = lo || (!hi && z <= KZ);
                        const bool keep = lo || hi || z <= KZ || z >= MZ - KZ;
                        const int mi = keep ? (in_lo ? z + KZ : z - MZ + KZ) : KZ;
                        const C r = field(mi);
                        v[n1] = keep ? r : f2(0.f, 0.f);
                    }
                };
                SFor<0, Z1>::run(ld);
                Dft<Z1, +1, C>::run(v);
#pragma unroll
                for (int k1 = 0; k1 < Z1; ++k1) X[k1 * ZR + t] = k1 == 0 ? v[0] : mul(v[k1], conjf2(twz[t * k1]));
            }
            __syncwarp();
            if (act && t < Z1) {
                C o[Z2];
#pragma unroll
                for (int n2 = 0; n2 < Z2; ++n2) o[n2] = X[t * ZR + n2];
                Dft<Z2, +1, C>::run(o);
                C* col = COL + f * CFS + n;
#pragma unroll
                for (int k2 = 0; k2 < Z2; ++k2) col[zrow<MX, MZ>(t + Z1 * k2) * S] = o[k2];
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // inverse x transform of the line pair (rows p, p + HP) of a column field;
    // dx: times i kx.  Threads t < X1 return x = t + X1 k2 in o[k2], row p in
    // .x and row p + HP in .y.
    auto xinv = [&](const C* src, int p, bool dx, int t, bool act, C* X, C* o) {
        const C* A0 = src + zrow<MX, MZ>(p) * S;
        const C* A1 = src + zrow<MX, MZ>(p + HP) * S;
        if (act && t < X2) {
            C v[X1];
            // slot n1 holds k = X2 n1 + t; the line is a + i b with a, b the two
            // rows: a_k + i b_k for k <= Kx, conj(a) + i conj(b) at Mx - k, the
            // Hermitian part (Re a_0, Re b_0) at k = 0 (and 0 for d_x)
            auto ld = [&](auto ic) {
                constexpr int n1 = decltype(ic)::value, k0 = X2 * n1, k1 = k0 + X2 - 1;
                constexpr bool lo = k1 <= KX, hi = k0 >= MX - KX, pad = k0 > KX && k1 < MX - KX;
                if constexpr (pad) {
                    v[n1] = f2(0.f, 0.f);
                } else {
                    const int k = k0 + t;
                    const bool in_lo = lo || (!hi && k <= KX);
                    const bool keep = lo || hi || k <= KX || k >= MX - KX;
                    const int kc = keep ? (in_lo ? k : MX - k) : 0;
                    C a = A0[kc], b = A1[kc];
                    if (dx) { const float kx = kxs[kc]; a = f2(-kx * a.y, kx * a.x); b = f2(-kx * b.y, kx * b.x); }
                    C Z = in_lo ? f2(a.x - b.y, a.y + b.x) : f2(a.x + b.y, b.x - a.y);
                    if (n1 == 0 && t == 0) Z = f2(a.x, b.x);
                    v[n1] = keep ? Z : f2(0.f, 0.f);
                }
            };
            SFor<0, X1>::run(ld);
            Dft<X1, +1, C>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < X1; ++k1) X[k1 * XR + t] = k1 == 0 ? v[0] : mul(v[k1], conjf2(twx[t * k1]));
        }
        __syncwarp();
        if (act && t < X1) {
#pragma unroll
            for (int n2 = 0; n2 < X2; ++n2) o[n2] = X[t * XR + n2];
            Dft<X2, +1, C>::run(o);
        }
        __syncwarp();
    };

    const int tx = lane / UX, gx = lane % UX;
    C* XX = XCH + (warp * UX + gx) * RSX;

    // ---- phase 2a: velocities into physical planes [f][x][z]
    for (int u0 = warp * UX; u0 < K::NU2; u0 += K::NSX) {
        const int u = u0 + gx;
        const bool act = u < K::NU2;
        const int f = act ? u / HP : 0, p = act ? u - f * HP : 0;
        C o[X2];
        xinv(COL + f * CFS, p, false, tx, act, XX, o);
        if (act && tx < X1) {
            float* dst = PLN + f * MX * MZP + p;
#pragma unroll
            for (int k2 = 0; k2 < X2; ++k2) {
                const int x = tx + X1 * k2;
                dst[x * MZP] = o[k2].x;
                dst[x * MZP + HP] = o[k2].y;
            }
        }
    }
    __syncthreads();

    // ---- phase 2b: products and forward x transforms, line pair (i, p); the
    // groups of component 0 also sum u v, those of component 2 w v (float-float)
    float uv_hi = 0.f, uv_lo = 0.f, wv_hi = 0.f, wv_lo = 0.f;
    const float sx = 1.0f / MX;
    for (int u0 = warp * UX; u0 < K::NU2; u0 += K::NSX) {
        const int u = u0 + gx;
        const bool act = u < K::NU2;
        const int i = act ? u / HP : 0, p = act ? u - i * HP : 0;
        C acc[X2];
#pragma unroll
        for (int k2 = 0; k2 < X2; ++k2) acc[k2] = f2(0.f, 0.f);
        // advective: N_i = sum_j u_j d_j u_i (d_x from the columns of u_i times
        // i kx); rotational: N_i = u_a omega_b - u_b omega_a with
        // (a, b) = (i + 2, i + 1) mod 3
        constexpr int NTERM = ROT ? 2 : 3;
#pragma unroll 1
        for (int j = 0; j < NTERM; ++j) {
            C o[X2];
            int src, vel;
            float sgn = 1.f;
            if (ROT) {
                const int a = (i + 2) % 3, b = (i + 1) % 3;
                src = 3 + (j == 0 ? b : a);
                vel = j == 0 ? a : b;
                sgn = j == 0 ? 1.f : -1.f;
            } else {
                src = j == 0 ? i : 3 * j + i;
                vel = j;
            }
            xinv(COL + src * CFS, p, !ROT && j == 0, tx, act, XX, o);
            if (act && tx < X1) {
                const float* pj = PLN + vel * MX * MZP + p;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) {
                    const int x = tx + X1 * k2;
                    acc[k2].x += (sgn * pj[x * MZP]) * o[k2].x;
                    acc[k2].y += (sgn * pj[x * MZP + HP]) * o[k2].y;
                }
            }
        }
        if (act && tx < X1 && i != 1) {
            const float* pa = PLN + i * MX * MZP + p;     // u or w
            const float* pv = PLN + MX * MZP + p;
#pragma unroll
            for (int k2 = 0; k2 < X2; ++k2) {
                const int o0 = (tx + X1 * k2) * MZP, o1 = o0 + HP;
                if (i == 0) {
                    ff_add_prod(uv_hi, uv_lo, pa[o0], pv[o0]);
                    ff_add_prod(uv_hi, uv_lo, pa[o1], pv[o1]);
                } else {
                    ff_add_prod(wv_hi, wv_lo, pa[o0], pv[o0]);
                    ff_add_prod(wv_hi, wv_lo, pa[o1], pv[o1]);
                }
            }
        }
        // forward x transform from the registers: x = tx + X1 k2, K = K1 + X2 K2
        if (act && tx < X1) {
            Dft<X2, -1, C>::run(acc);
#pragma unroll
            for (int k1 = 0; k1 < X2; ++k1) XX[k1 * XRF + tx] = k1 == 0 ? acc[0] : mul(acc[k1], twx[tx * k1]);
        }
        __syncwarp();
        C zk[X1];
        if (act && tx < X2) {
#pragma unroll
            for (int n2 = 0; n2 < X1; ++n2) zk[n2] = XX[tx * XRF + n2];
            Dft<X1, -1, C>::run(zk);
        }
        __syncwarp();
        if (act && tx < X2) {
#pragma unroll
            for (int k2 = 0; k2 < X1; ++k2) XX[tx + X2 * k2] = zk[k2];
        }
        __syncwarp();
        // split the two real rows, keep kx <= Kx, scale 1/Mx
        if (act) {
            C* R0 = COL + i * CFS + zrow<MX, MZ>(p) * S;
            C* R1 = COL + i * CFS + zrow<MX, MZ>(p + HP) * S;
            for (int n = tx; n <= KX; n += GX) {
                const C Zn = XX[n], Zc = XX[(MX - n) % MX];
                R0[n] = f2(0.5f * (Zn.x + Zc.x) * sx, 0.5f * (Zn.y - Zc.y) * sx);
                R1[n] = f2(0.5f * (Zn.y + Zc.y) * sx, 0.5f * (Zc.x - Zn.x) * sx);
            }
        }
        __syncwarp();
    }
    // plane means <uv>, <wv>
    {
        double suv = 0.0, swv = 0.0;
        ff_block_sum2(uv_hi, uv_lo, wv_hi, wv_lo, (float*)red, &suv, &swv);
        if (tid == 0) {
            g.uv[(size_t)e * My + y + 1] = suv / (double)K::PLANE;
            g.wv[(size_t)e * My + y + 1] = swv / (double)K::PLANE;
        }
    }

    // ---- phase 3: forward z transforms of the kept columns, truncation
    {
        const int t = lane / UZ, gi = lane % UZ;
        C* X = XCH + (warp * UZ + gi) * RSZ;
        C* N3 = (C*)g.N3;
        const float sz = 1.0f / MZ;
        for (int u0 = warp * UZ; u0 < K::NU3; u0 += K::NSZ) {
            const int u = u0 + gi;
            const bool act = u < K::NU3;
            const int i = act ? u / NKX : 0, n = act ? u - i * NKX : 0;
            if (act && t < Z2) {
                const C* col = COL + i * CFS + n;
                C v[Z1];
#pragma unroll
                for (int n1 = 0; n1 < Z1; ++n1) v[n1] = col[zrow<MX, MZ>(Z2 * n1 + t) * S];
                Dft<Z1, -1, C>::run(v);
#pragma unroll
                for (int k1 = 0; k1 < Z1; ++k1) X[k1 * ZR + t] = k1 == 0 ? v[0] : mul(v[k1], twz[t * k1]);
            }
            __syncwarp();
            if (act && t < Z1) {
                C o[Z2];
#pragma unroll
                for (int n2 = 0; n2 < Z2; ++n2) o[n2] = X[t * ZR + n2];
                Dft<Z2, -1, C>::run(o);
                C* out = N3 + (size_t)i * fs + off0 + n;
#pragma unroll
                for (int k2 = 0; k2 < Z2; ++k2) {
                    const int m = t + Z1 * k2;
                    const int mi = m <= KZ ? m + KZ : (m >= MZ - KZ ? m - MZ + KZ : -1);
                    if (mi >= 0) out[mi * NKX] = f2(o[k2].x * sz, o[k2].y * sz);
                }
            }
            __syncwarp();
        }
    }
}

template <int MX, int MZ, bool ROT>
void launch_t(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
    typedef LCfg<MX, MZ, ROT> K;
    k_plane_lines<MX, MZ, ROT><<<dim3(g.ny, g.E), K::NT, K::BYTES, st>>>(g, U, W);
}

template <int MX, int MZ>
void set_attr_t() {
    static_assert(LCfg<MX, MZ, false>::BYTES <= 227 * 1024, "plane stage does not fit in shared memory");
    static_assert(LCfg<MX, MZ, true>::BYTES <= 227 * 1024, "plane stage does not fit in shared memory");
    cudaFuncSetAttribute(k_plane_lines<MX, MZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)LCfg<MX, MZ, false>::BYTES);
    cudaFuncSetAttribute(k_plane_lines<MX, MZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)LCfg<MX, MZ, true>::BYTES);
}

}  // namespace pln

#define DNS_LINES_SIZES(X) X(16, 16) X(16, 32) X(16, 48) X(16, 64) X(32, 16) X(32, 32) X(32, 48) X(32, 64) \
    X(48, 16) X(48, 32) X(48, 48) X(48, 64) X(64, 16) X(64, 32) X(64, 48) X(64, 64)

bool launch_plane_lines(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
#define DNS_CASE(a, b)                                                   \
    if (g.mx == a && g.mz == b) {                                        \
        if (g.rot) pln::launch_t<a, b, true>(g, U, W, st);               \
        else pln::launch_t<a, b, false>(g, U, W, st);                    \
        return true;                                                     \
    }
    DNS_LINES_SIZES(DNS_CASE)
#undef DNS_CASE
    return false;
}

size_t plane_lines_smem_bytes(int mx, int mz) {
#define DNS_CASE(a, b) if (mx == a && mz == b) return pln::LCfg<a, b, false>::BYTES;
    DNS_LINES_SIZES(DNS_CASE)
#undef DNS_CASE
    return 0;
}

void set_attributes_plane_lines() {
#define DNS_CASE(a, b) pln::set_attr_t<a, b>();
    DNS_LINES_SIZES(DNS_CASE)
#undef DNS_CASE
}

}  // namespace dnsk
