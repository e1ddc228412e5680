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
#include "dns_internal.hpp"
#include "dft.cuh"

namespace dnsk {

namespace pln {

using namespace dft;
typedef float2 C;

__device__ __forceinline__ C f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ C conjf2(C a) { return make_float2(a.x, -a.y); }

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

template <int MX, int MZ>
struct LCfg {
    static constexpr int KX = (MX - 1) / 3, KZ = (MZ - 1) / 3;
    static constexpr int NKX = KX + 1, NKZ = 2 * KZ + 1, NM = NKX * NKZ;
    static constexpr int X1 = Split<MX>::N1, X2 = Split<MX>::N2;
    static constexpr int Z1 = Split<MZ>::N1, Z2 = Split<MZ>::N2;
    static constexpr int GX = cmax(X1, X2), GZ = cmax(Z1, Z2);   // threads per line
    static constexpr int UX = 32 / GX, UZ = 32 / GZ;              // lines per warp
    static constexpr int HP = MZ / 2;                             // line pairs
    static constexpr int NU1 = 9 * NKX, NU2 = 3 * HP, NU3 = 3 * NKX;
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
    static constexpr size_t B_PLN = al16(B_COL + sizeof(C) * 9 * CFS);
    static constexpr size_t PLN_BYTES = smax(sizeof(float) * 3 * MX * MZP, sizeof(C) * 5 * NKZ * NKXB);
    static constexpr size_t B_X = al16(B_PLN + PLN_BYTES);
    static constexpr size_t B_TW = al16(B_X + sizeof(C) * smax((size_t)NSX * RSX, (size_t)NSZ * RSZ));
    static constexpr size_t B_K = B_TW + sizeof(C) * (MX + MZ);
    static constexpr size_t B_RED = al16(B_K + sizeof(float) * (NKX + NKZ + NKZ * NKXB));
    static constexpr size_t BYTES = B_RED + (2 + 2 * 32) * sizeof(double);
    static constexpr int MINB = (2 * (BYTES + 1024) <= 228 * 1024 && NT * 2 * 64 <= 65536) ? 2 : 1;
    static_assert(MZ % 8 == 0, "z-row permutation works in blocks of eight");
};

template <int MX, int MZ>
__device__ __forceinline__ int zrow(int z) {
    if (!LCfg<MX, MZ>::PERM) return z;
    const int b = z & 7;
    return (z & ~7) | ((2 * b) & 7) | (b >> 2);
}

template <int MX, int MZ>
__global__ void __launch_bounds__(LCfg<MX, MZ>::NT, LCfg<MX, MZ>::MINB)
k_plane_lines(GroupView g, const double* __restrict__ Ucur, const double* __restrict__ Wcur) {
    typedef LCfg<MX, MZ> K;
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

    // ---- stage inputs [f][m][n] (padded rows) and tables
    {
        const C* P = (const C*)g.P5;
        for (int i = tid; i < 5 * NM; i += NT) {
            const int f = i / NM, q = i - f * NM, mi = q / NKX, n = q - mi * NKX;
            BASE[f * FSB + mi * NKXB + n] = P[f * fs + off0 + q];
        }
        for (int i = tid; i < MX; i += NT) twx[i] = g.twxf[i];
        for (int i = tid; i < MZ; i += NT) twz[i] = g.twzf[i];
        for (int i = tid; i < NKX; i += NT) kxs[i] = g.kxtf[i];
        for (int i = tid; i < NKZ; i += NT) kzs[i] = g.kztf[i];
        for (int q = tid; q < NM; q += NT) {
            const int mi = q / NKX;
            k2s[mi * NKXB + q - mi * NKX] = g.k2invf[q];
        }
    }
    const float Um = (float)Ucur[(size_t)e * My + y + 1];
    const float Wm = (float)Wcur[(size_t)e * My + y + 1];
    mean_dy_row(g.D1, Ucur + (size_t)e * My, Wcur + (size_t)e * My, My, y + 1, red);
    __syncthreads();
    const float dUm = (float)red[0];
    const float dWm = (float)red[1];

    // spectral value at mode (mi, n) of u_comp (kind 0), d_y u_comp (kind 1)
    // or d_z u_comp (kind 2); u, w from v, eta as u = i (kx Dv - kz eta) / k^2,
    // w = i (kz Dv + kx eta) / k^2, the (0, 0) mode from the mean flow
    auto gen = [&](int kind, int comp, int mi, int n) -> C {
        const C* B = BASE + mi * NKXB + n;
        const bool mean = (mi == KZ && n == 0);
        if (kind == 1) {
            if (comp == 1) return B[FSB];
            if (mean) return f2(comp == 0 ? dUm : dWm, 0.f);
            const float kx = kxs[n], kz = kzs[mi], ki = k2s[mi * NKXB + n];
            const C d2 = B[2 * FSB], de = B[4 * FSB];
            float ax, ay;
            if (comp == 0) { ax = (kx * d2.x - kz * de.x) * ki; ay = (kx * d2.y - kz * de.y) * ki; }
            else { ax = (kz * d2.x + kx * de.x) * ki; ay = (kz * d2.y + kx * de.y) * ki; }
            return f2(-ay, ax);
        }
        C b;
        if (comp == 1) {
            b = B[0];
        } else if (mean) {
            b = f2(comp == 0 ? Um : Wm, 0.f);
        } else {
            const float kx = kxs[n], kz = kzs[mi], ki = k2s[mi * NKXB + n];
            const C dv = B[FSB], et = B[3 * FSB];
            float ax, ay;
            if (comp == 0) { ax = (kx * dv.x - kz * et.x) * ki; ay = (kx * dv.y - kz * et.y) * ki; }
            else { ax = (kz * dv.x + kx * et.x) * ki; ay = (kz * dv.y + kx * et.y) * ki; }
            b = f2(-ay, ax);
        }
        if (kind == 0) return b;
        const float kz = kzs[mi];
        return f2(-kz * b.y, kz * b.x);
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
            if (act && t < Z2) {
                C v[Z1];
#pragma unroll
                for (int n1 = 0; n1 < Z1; ++n1) {
                    const int z = Z2 * n1 + t;
                    const int mi = z <= KZ ? z + KZ : (z >= MZ - KZ ? z - MZ + KZ : -1);
                    v[n1] = mi >= 0 ? gen(kind, comp, mi, n) : f2(0.f, 0.f);
                }
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
#pragma unroll
            for (int n1 = 0; n1 < X1; ++n1) {
                const int k = X2 * n1 + t;
                C Z = f2(0.f, 0.f);
                if (k == 0) {
                    if (!dx) Z = f2(A0[0].x, A1[0].x);          // Hermitian part of the kx = 0 column
                } else if (k <= KX) {
                    C a = A0[k], b = A1[k];
                    if (dx) { const float kx = kxs[k]; a = f2(-kx * a.y, kx * a.x); b = f2(-kx * b.y, kx * b.x); }
                    Z = f2(a.x - b.y, a.y + b.x);               // a + i b
                } else if (k >= MX - KX) {
                    C a = A0[MX - k], b = A1[MX - k];
                    if (dx) { const float kx = kxs[MX - k]; a = f2(-kx * a.y, kx * a.x); b = f2(-kx * b.y, kx * b.x); }
                    Z = f2(a.x + b.y, b.x - a.y);               // conj(a) + i conj(b)
                }
                v[n1] = Z;
            }
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

    // ---- phase 2b: products and forward x transforms, line pair (i, p)
    double s_uv = 0.0, s_wv = 0.0;
    const float sx = 1.0f / MX;
    for (int u0 = warp * UX; u0 < K::NU2; u0 += K::NSX) {
        const int u = u0 + gx;
        const bool act = u < K::NU2;
        const int i = act ? u / HP : 0, p = act ? u - i * HP : 0;
        C acc[X2];
#pragma unroll
        for (int k2 = 0; k2 < X2; ++k2) acc[k2] = f2(0.f, 0.f);
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            C o[X2];
            xinv(COL + (j == 0 ? i : 3 * j + i) * CFS, p, j == 0, tx, act, XX, o);
            if (act && tx < X1) {
                const float* pj = PLN + j * MX * MZP + p;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) {
                    const int x = tx + X1 * k2;
                    acc[k2].x += pj[x * MZP] * o[k2].x;
                    acc[k2].y += pj[x * MZP + HP] * o[k2].y;
                }
            }
        }
        if (act && tx < X1 && i == 0) {
            const float* pu = PLN + p;
            const float* pv = pu + MX * MZP;
            const float* pw = pv + MX * MZP;
#pragma unroll
            for (int k2 = 0; k2 < X2; ++k2) {
                const int o0 = (tx + X1 * k2) * MZP, o1 = o0 + HP;
                s_uv += (double)pu[o0] * (double)pv[o0] + (double)pu[o1] * (double)pv[o1];
                s_wv += (double)pw[o0] * (double)pv[o0] + (double)pw[o1] * (double)pv[o1];
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
    // plane means: warp sums, then a fixed-order sum over warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_uv += __shfl_xor_sync(0xffffffffu, s_uv, o);
        s_wv += __shfl_xor_sync(0xffffffffu, s_wv, o);
    }
    if (lane == 0) {
        red[2 + 2 * warp] = s_uv;
        red[3 + 2 * warp] = s_wv;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < K::NW; ++w) { a += red[2 + 2 * w]; b += red[3 + 2 * w]; }
        g.uv[(size_t)e * My + y + 1] = a / (double)K::PLANE;
        g.wv[(size_t)e * My + y + 1] = b / (double)K::PLANE;
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

template <int MX, int MZ>
void launch_t(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
    typedef LCfg<MX, MZ> K;
    k_plane_lines<MX, MZ><<<dim3(g.ny, g.E), K::NT, K::BYTES, st>>>(g, U, W);
}

template <int MX, int MZ>
void set_attr_t() {
    typedef LCfg<MX, MZ> K;
    static_assert(K::BYTES <= 227 * 1024, "plane stage does not fit in shared memory");
    cudaFuncSetAttribute(k_plane_lines<MX, MZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::BYTES);
}

}  // namespace pln

#define DNS_LINES_SIZES(X) X(16, 16) X(16, 32) X(16, 48) X(16, 64) X(32, 16) X(32, 32) X(32, 48) X(32, 64) \
    X(48, 16) X(48, 32) X(48, 48) X(48, 64) X(64, 16) X(64, 32) X(64, 48) X(64, 64)

bool launch_plane_lines(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
#define DNS_CASE(a, b) if (g.mx == a && g.mz == b) { pln::launch_t<a, b>(g, U, W, st); return true; }
    DNS_LINES_SIZES(DNS_CASE)
#undef DNS_CASE
    return false;
}

size_t plane_lines_smem_bytes(int mx, int mz) {
#define DNS_CASE(a, b) if (mx == a && mz == b) return pln::LCfg<a, b>::BYTES;
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
