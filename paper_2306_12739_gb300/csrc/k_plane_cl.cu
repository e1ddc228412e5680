// Physical-space stage of one sub-step (paper Sec. 3.1-3.2) for one interior
// y-plane of one member, split over a thread-block cluster of CL CTAs so that
// large planes fit on chip and small ones leave room for two CTAs per SM.
// Same mathematics as k_plane.cu: u, w from v, eta; 12 inverse transforms
// with 2/3-rule zero padding; N_i = u_j d_j u_i; plane means <uv>, <wv>;
// 3 forward transforms with truncation.
//
// Work split inside the cluster (rank r):
//   * z transforms: rank r owns the kept columns n in [r NKL, (r+1) NKL); it
//     transforms them over all Mz rows and delivers each row to the rank that
//     owns it, straight into that rank's shared memory (distributed shared
//     memory stores, then a cluster barrier);
//   * x transforms and the pointwise products: rank r owns the line pairs
//     p in [r HPL, (r+1) HPL), i.e. rows p and p + Mz/2;
//   * forward: x transforms on the owned rows, then each kept column goes to
//     its column owner for the z transform and truncation.
// Every 1-D transform is a four-step N1 x N2 FFT with in-register DFTs.  No
// atomics: the plane means are combined in a fixed order by rank 0.
#include "dns_internal.hpp"
#include "dft.cuh"
#include "ff.cuh"
#include <type_traits>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace dnsk {

namespace pcl {

using namespace dft;


template <typename T, int MX, int MZ, int CL>
struct Cfg {
    typedef typename Cx<T>::t C;
    static constexpr int KX = (MX - 1) / 3, KZ = (MZ - 1) / 3;
    static constexpr int NKX = KX + 1, NKZ = 2 * KZ + 1, NM = NKX * NKZ;
    static constexpr int NKXP = NKX | 1;
    static constexpr int X1 = Split<MX>::N1, X2 = Split<MX>::N2;
    static constexpr int Z1 = Split<MZ>::N1, Z2 = Split<MZ>::N2;
    static constexpr int HP = MZ / 2;            // line pairs of a whole plane
    static constexpr int HPL = HP / CL;          // line pairs of one rank
    static constexpr int ZL = 2 * HPL;           // rows of one rank
    static constexpr int NKL = (NKX + CL - 1) / CL;   // columns of one rank
    static constexpr int NKLP = NKL | 1;
    static constexpr int NF = 3;
    static constexpr int PL = MX * ZL;           // points of one rank
    static constexpr int AS = ZL * NKXP;         // inverse column slot [zl][n]
    static constexpr int AF = MZ * NKLP;         // forward column slot [z][nl]
    static constexpr int SSP = cmax(cmax(Z1 * Z2 * NKLP, X1 * X2 * HPL), MX * HPL);
    static constexpr int NT0 = NF * HPL * X2;
    static constexpr int NT = ((NT0 + 31) / 32) * 32;
    static constexpr size_t CB = sizeof(C), TB = sizeof(T);
    static constexpr size_t B_BASE = 0;                                  // C [5][NKZ][NKL]
    static constexpr size_t B_PLN = B_BASE + CB * 5 * NKZ * NKL;        // T [3][MX][ZL]
    static constexpr size_t B_A = ((B_PLN + TB * 3 * PL) + 15) / 16 * 16;   // C [6][AS]
    static constexpr size_t B_F = B_A + CB * 6 * AS;                     // C [AF]
    static constexpr size_t B_S = B_F + CB * AF;                         // C [NF][SSP]
    static constexpr size_t B_TW = B_S + CB * NF * SSP;                  // C [MX + MZ]
    static constexpr size_t B_K = B_TW + CB * (MX + MZ);                 // T [NKX + NKZ + NKZ*NKL]
    static constexpr size_t B_RED = ((B_K + TB * (NKX + NKZ + NKZ * NKL)) + 15) / 16 * 16;  // double [64 + 2 CL]
    static constexpr size_t BYTES = B_RED + sizeof(double) * (64 + 2 * CL);
    // two CTAs per SM where shared memory allows it (registers capped to match)
    static constexpr int MINB = (2 * BYTES <= 227 * 1024 && NT <= 512) ? 2 : 1;
    static_assert(HP % CL == 0, "line pairs must split evenly over the cluster");
    static_assert(NF * HPL * X1 <= NT, "one x-stage step-C task per thread");
    static_assert(NT <= 1024, "too many threads");
};

template <typename T, int MX, int MZ, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(Cfg<T, MX, MZ, CL>::NT, Cfg<T, MX, MZ, CL>::MINB)
k_plane_cl(GroupView g, const double* __restrict__ Ucur, const double* __restrict__ Wcur) {
    typedef Cfg<T, MX, MZ, CL> K;
    typedef typename K::C C;
    constexpr int KX = K::KX, KZ = K::KZ, NKX = K::NKX, NKZ = K::NKZ, NM = K::NM, NKXP = K::NKXP;
    constexpr int X1 = K::X1, X2 = K::X2, Z1 = K::Z1, Z2 = K::Z2, HP = K::HP, HPL = K::HPL, ZL = K::ZL;
    constexpr int NKL = K::NKL, NKLP = K::NKLP, NF = K::NF, PL = K::PL, AS = K::AS, SSP = K::SSP, NT = K::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rk = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int y = blockIdx.x / CL, e = blockIdx.y, E = g.E, Ny = g.ny, My = g.my;
    const int pl0 = rk * HPL;                 // first owned line pair
    const int c0 = rk * NKL;                  // first owned column
    const int nc = NKX - c0 < NKL ? NKX - c0 : NKL;
    const size_t fs = (size_t)Ny * E * NM;
    const size_t off0 = ((size_t)y * E + e) * NM;

    C* base = (C*)(smem + K::B_BASE);
    T* pl = (T*)(smem + K::B_PLN);
    T* PU = pl;
    T* PV = pl + PL;
    T* PW = pl + 2 * PL;
    C* Ainv = (C*)(smem + K::B_A);
    C* Afwd = (C*)(smem + K::B_F);
    C* Sb = (C*)(smem + K::B_S);
    C* twx = (C*)(smem + K::B_TW);
    C* twz = twx + MX;
    T* kxs = (T*)(smem + K::B_K);
    T* kzs = kxs + NKX;
    T* k2s = kzs + NKZ;                       // [NKZ][NKL]
    double* red = (double*)(smem + K::B_RED); // [64] block reductions, then [2 CL] cluster partials

    // ---- stage the owned columns of the five spectral inputs and the tables
    {
        const C* P = (const C*)g.P5;
        for (int i = tid; i < 5 * NKZ * NKL; i += NT) {
            const int f = i / (NKZ * NKL), r = i - f * (NKZ * NKL), mi = r / NKL, nl = r - mi * NKL;
            C v = mk<C>((T)0, (T)0);
            if (nl < nc) v = P[f * fs + off0 + (size_t)mi * NKX + c0 + nl];
            base[i] = v;
        }
        const C* tx = (const C*)(sizeof(T) == 8 ? (const void*)g.twx : (const void*)g.twxf);
        const C* tz = (const C*)(sizeof(T) == 8 ? (const void*)g.twz : (const void*)g.twzf);
        for (int i = tid; i < MX; i += NT) twx[i] = tx[i];
        for (int i = tid; i < MZ; i += NT) twz[i] = tz[i];
        for (int i = tid; i < NKX; i += NT) kxs[i] = (T)g.kxt[i];
        for (int i = tid; i < NKZ; i += NT) kzs[i] = (T)g.kzt[i];
        for (int i = tid; i < NKZ * NKL; i += NT) {
            const int mi = i / NKL, nl = i - mi * NKL;
            k2s[i] = nl < nc ? (T)g.k2inv[mi * NKX + c0 + nl] : (T)0;
        }
    }
    mean_dy_row(g.D1, Ucur + (size_t)e * My, Wcur + (size_t)e * My, My, y + 1, red);
    const T Um = (T)Ucur[(size_t)e * My + y + 1];
    const T Wm = (T)Wcur[(size_t)e * My + y + 1];
    __syncthreads();
    const T dUm = (T)red[0];
    const T dWm = (T)red[1];
    __syncthreads();
    const C* Bv = base;
    const C* BDv = base + NKZ * NKL;
    const C* BD2v = base + 2 * NKZ * NKL;
    const C* Be = base + 3 * NKZ * NKL;
    const C* BDe = base + 4 * NKZ * NKL;

    // spectral value of field `which` at (mi, owned column nl):
    // 0 u, 1 v, 2 w, 3 + 3 i + j = d u_i / d x_j
    auto gen = [&](int which, int mi, int nl) -> C {
        const int n = c0 + nl, b = mi * NKL + nl;
        const T kx = kxs[n], kz = kzs[mi], ki = k2s[b];
        const bool mean = (mi == KZ && n == 0);
        const int comp = which < 3 ? which : (which - 3) / 3;
        const int dir = which < 3 ? -1 : (which - 3) % 3;
        if (dir == 1) {
            if (comp == 1) return BDv[b];
            if (mean) return mk<C>(comp == 0 ? dUm : dWm, (T)0);
            const C d2 = BD2v[b], de = BDe[b];
            T ax, ay;
            if (comp == 0) { ax = (kx * d2.x - kz * de.x) * ki; ay = (kx * d2.y - kz * de.y) * ki; }
            else { ax = (kz * d2.x + kx * de.x) * ki; ay = (kz * d2.y + kx * de.y) * ki; }
            return mk<C>(-ay, ax);
        }
        C bb;
        if (comp == 1) {
            bb = Bv[b];
        } else if (mean) {
            bb = mk<C>(comp == 0 ? Um : Wm, (T)0);
        } else {
            const C dv = BDv[b], et = Be[b];
            T ax, ay;
            if (comp == 0) { ax = (kx * dv.x - kz * et.x) * ki; ay = (kx * dv.y - kz * et.y) * ki; }
            else { ax = (kz * dv.x + kx * et.x) * ki; ay = (kz * dv.y + kx * et.y) * ki; }
            bb = mk<C>(-ay, ax);
        }
        if (dir < 0) return bb;
        const T k = dir == 0 ? kx : kz;
        return mk<C>(-k * bb.y, k * bb.x);
    };

    // ---- inverse transforms of three fields.  mode 0 (u, v, w): into PU/PV/PW,
    // their z-transformed rows kept in A slots 3..5; mode 1 (the derivatives of
    // component xc): into the scratch slots as [x][pl] packed line pairs; the x
    // derivative reuses u_xc's kept rows times i kx and needs no z transform.
    auto inverse3 = [&](int w0, int w1, int w2, int mode, int xc) {
        const int f_lo = (mode == 1) ? 1 : 0;
        auto aslot = [&](int f) -> C* { return Ainv + (mode == 0 ? 3 + f : f) * AS; };
        // z-stage step A on the owned columns: tasks (f, n2, nl), nl fastest
        for (int t = tid; t < (NF - f_lo) * NKL * Z2; t += NT) {
            const int nl = t % NKL, r = t / NKL, n2 = r % Z2, f = f_lo + r / Z2;
            if (nl >= nc) continue;
            const int which = f == 0 ? w0 : (f == 1 ? w1 : w2);
            C v[Z1];
#pragma unroll
            for (int n1 = 0; n1 < Z1; ++n1) {
                const int z = Z2 * n1 + n2;
                int mi = -1;
                if (z <= KZ) mi = z + KZ;
                else if (z >= MZ - KZ) mi = z - MZ + KZ;
                v[n1] = mi >= 0 ? gen(which, mi, nl) : mk<C>((T)0, (T)0);
            }
            Dft<Z1, +1, C>::run(v);
            C* S = Sb + f * SSP + n2 * NKLP + nl;
#pragma unroll
            for (int k1 = 0; k1 < Z1; ++k1) {
                const C w = twz[n2 * k1];
                S[k1 * (Z2 * NKLP)] = k1 == 0 ? v[0] : mul(v[k1], mk<C>(w.x, -w.y));
            }
        }
        // The scratch rows just written are read by other threads of this CTA in
        // step C: a CTA barrier orders them.  Across the cluster, every rank has
        // also finished reading its A slots of the previous transform (their values
        // consumed before its last CTA barrier) and, in the first transform, has
        // started: an execution barrier of the cluster suffices for that, without
        // the release of this rank's writes that a default cluster barrier costs.
        __syncthreads();
        asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
        // z-stage step C: tasks (f, k1, nl); row z goes to the rank owning it
        for (int t = tid; t < (NF - f_lo) * NKL * Z1; t += NT) {
            const int nl = t % NKL, r = t / NKL, k1 = r % Z1, f = f_lo + r / Z1;
            if (nl >= nc) continue;
            const C* S = Sb + f * SSP + k1 * (Z2 * NKLP) + nl;
            C v[Z2];
#pragma unroll
            for (int n2 = 0; n2 < Z2; ++n2) v[n2] = S[n2 * NKLP];
            Dft<Z2, +1, C>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < Z2; ++k2) {
                const int z = k1 + Z1 * k2;
                const int up = z >= HP ? 1 : 0;
                const int p = z - up * HP;
                const int owner = p / HPL, zl = up * HPL + (p - owner * HPL);
                C* dst = cluster.map_shared_rank(aslot(f), owner);
                dst[zl * NKXP + c0 + nl] = v[k2];
            }
        }
        cluster.sync();
        // x-stage step A on the owned line pairs: tasks (f, n2, pl), pl fastest
        for (int t = tid; t < NF * HPL * X2; t += NT) {
            const int p = t % HPL, r = t / HPL, n2 = r % X2, f = r / X2;
            const bool dx = (f == 0 && mode == 1);
            const C* A0 = (dx ? Ainv + (3 + xc) * AS : aslot(f)) + p * NKXP;
            const C* A1 = A0 + HPL * NKXP;
            C v[X1];
#pragma unroll
            for (int n1 = 0; n1 < X1; ++n1) {
                const int k = X2 * n1 + n2;
                C Z = mk<C>((T)0, (T)0);
                if (k == 0) {
                    if (!dx) Z = mk<C>(A0[0].x, A1[0].x);      // Hermitian part of the n = 0 column
                } else if (k <= KX) {
                    C a = A0[k], b = A1[k];
                    if (dx) { const T kx = kxs[k]; a = mk<C>(-kx * a.y, kx * a.x); b = mk<C>(-kx * b.y, kx * b.x); }
                    Z = mk<C>(a.x - b.y, a.y + b.x);           // a + i b
                } else if (k >= MX - KX) {
                    C a = A0[MX - k], b = A1[MX - k];
                    if (dx) { const T kx = kxs[MX - k]; a = mk<C>(-kx * a.y, kx * a.x); b = mk<C>(-kx * b.y, kx * b.x); }
                    Z = mk<C>(a.x + b.y, b.x - a.y);           // conj(a) + i conj(b)
                }
                v[n1] = Z;
            }
            Dft<X1, +1, C>::run(v);
            C* S = Sb + f * SSP + n2 * HPL + p;
#pragma unroll
            for (int k1 = 0; k1 < X1; ++k1) {
                const C w = twx[n2 * k1];
                S[k1 * (X2 * HPL)] = k1 == 0 ? v[0] : mul(v[k1], mk<C>(w.x, -w.y));
            }
        }
        __syncthreads();
        // x-stage step C: one task (f, k1, pl) per thread
        C out[X2];
        const bool active = tid < NF * HPL * X1;
        int cf = 0, cp = 0, ck1 = 0;
        if (active) {
            cp = tid % HPL;
            const int r = tid / HPL;
            ck1 = r % X1;
            cf = r / X1;
            const C* S = Sb + cf * SSP + ck1 * (X2 * HPL) + cp;
#pragma unroll
            for (int n2 = 0; n2 < X2; ++n2) out[n2] = S[n2 * HPL];
            Dft<X2, +1, C>::run(out);
        }
        if (mode == 1) __syncthreads();     // the scratch is overwritten below
        if (active) {
            if (mode == 0) {
                T* dst = pl + cf * PL + cp;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) {
                    const int x = ck1 + X1 * k2;
                    dst[x * ZL] = out[k2].x;
                    dst[x * ZL + HPL] = out[k2].y;
                }
            } else {
                C* dst = Sb + cf * SSP + cp;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) dst[(ck1 + X1 * k2) * HPL] = out[k2];
            }
        }
        __syncthreads();
    };

    // ---- forward transform of the advective sum held in slot 0 as [x][pl]
    // packed line pairs; the owned kept modes go to global memory
    auto forward = [&](C* __restrict__ gout) {
        for (int t = tid; t < HPL * X2; t += NT) {
            const int p = t % HPL, n2 = t / HPL;
            C v[X1];
#pragma unroll
            for (int n1 = 0; n1 < X1; ++n1) v[n1] = Sb[(X2 * n1 + n2) * HPL + p];
            Dft<X1, -1, C>::run(v);
            C* S = Sb + SSP + n2 * HPL + p;
#pragma unroll
            for (int k1 = 0; k1 < X1; ++k1) S[k1 * (X2 * HPL)] = k1 == 0 ? v[0] : mul(v[k1], twx[n2 * k1]);
        }
        __syncthreads();
        for (int t = tid; t < HPL * X1; t += NT) {
            const int p = t % HPL, k1 = t / HPL;
            const C* S = Sb + SSP + k1 * (X2 * HPL) + p;
            C v[X2];
#pragma unroll
            for (int n2 = 0; n2 < X2; ++n2) v[n2] = S[n2 * HPL];
            Dft<X2, -1, C>::run(v);
            C* O = Sb + 2 * SSP + p;
#pragma unroll
            for (int k2 = 0; k2 < X2; ++k2) O[(k1 + X1 * k2) * HPL] = v[k2];
        }
        __syncthreads();
        // split the two real rows, keep n <= KX, scale 1/MX, send column n to its owner
        const T sx = (T)1 / (T)MX;
        for (int t = tid; t < HPL * NKX; t += NT) {
            const int p = t % HPL, n = t / HPL;
            const C* O = Sb + 2 * SSP + p;
            const C Zn = O[n * HPL], Zc = O[((MX - n) % MX) * HPL];
            const C xa = mk<C>((T)0.5 * (Zn.x + Zc.x) * sx, (T)0.5 * (Zn.y - Zc.y) * sx);
            const C xb = mk<C>((T)0.5 * (Zn.y + Zc.y) * sx, (T)0.5 * (Zc.x - Zn.x) * sx);
            const int owner = n / NKL, nl = n - owner * NKL;
            C* dst = cluster.map_shared_rank(Afwd, owner);
            dst[(pl0 + p) * NKLP + nl] = xa;
            dst[(HP + pl0 + p) * NKLP + nl] = xb;
        }
        cluster.sync();
        for (int t = tid; t < NKL * Z2; t += NT) {
            const int nl = t % NKL, n2 = t / NKL;
            if (nl >= nc) continue;
            C v[Z1];
#pragma unroll
            for (int n1 = 0; n1 < Z1; ++n1) v[n1] = Afwd[(Z2 * n1 + n2) * NKLP + nl];
            Dft<Z1, -1, C>::run(v);
            C* S = Sb + n2 * NKLP + nl;
#pragma unroll
            for (int k1 = 0; k1 < Z1; ++k1) S[k1 * (Z2 * NKLP)] = k1 == 0 ? v[0] : mul(v[k1], twz[n2 * k1]);
        }
        __syncthreads();
        C* stage = Sb + SSP;
        const T sz = (T)1 / (T)MZ;
        for (int t = tid; t < NKL * Z1; t += NT) {
            const int nl = t % NKL, k1 = t / NKL;
            if (nl >= nc) continue;
            const C* S = Sb + k1 * (Z2 * NKLP) + nl;
            C v[Z2];
#pragma unroll
            for (int n2 = 0; n2 < Z2; ++n2) v[n2] = S[n2 * NKLP];
            Dft<Z2, -1, C>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < Z2; ++k2) {
                const int m = k1 + Z1 * k2;
                int mi = -1;
                if (m <= KZ) mi = m + KZ;
                else if (m >= MZ - KZ) mi = m - MZ + KZ;
                if (mi >= 0) stage[mi * NKL + nl] = scal(v[k2], sz);
            }
        }
        __syncthreads();
        for (int i = tid; i < NKZ * NKL; i += NT) {
            const int mi = i / NKL, nl = i - mi * NKL;
            if (nl < nc) gout[(size_t)mi * NKX + c0 + nl] = stage[i];
        }
        __syncthreads();
    };

    // velocities
    inverse3(0, 1, 2, 0, -1);
    // plane means <uv>, <wv>: per-rank partial sums, combined by rank 0 in rank order
    {
        double s1 = 0.0, s2 = 0.0;
        if constexpr (std::is_same<T, float>::value) {
            // single precision: float-float sums (the FP64 pipe is slow)
            float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
            for (int i = tid; i < PL; i += NT) {
                ff_add_prod(h1, l1, PU[i], PV[i]);
                ff_add_prod(h2, l2, PW[i], PV[i]);
            }
            ff_block_sum2(h1, l1, h2, l2, (float*)red, &s1, &s2);
        } else {
            for (int i = tid; i < PL; i += NT) {
                s1 += (double)PU[i] * (double)PV[i];
                s2 += (double)PW[i] * (double)PV[i];
            }
            s1 = block_sum(s1, red);
            s2 = block_sum(s2, red);
        }
        if (tid == 0) {
            double* dst = cluster.map_shared_rank(red + 64, 0);
            dst[2 * rk] = s1;
            dst[2 * rk + 1] = s2;
        }
        cluster.sync();
        if (rk == 0 && tid == 0) {
            double a = 0.0, b = 0.0;
            for (int r = 0; r < CL; ++r) { a += red[64 + 2 * r]; b += red[64 + 2 * r + 1]; }
            g.uv[(size_t)e * My + y + 1] = a / (double)(MX * MZ);
            g.wv[(size_t)e * My + y + 1] = b / (double)(MX * MZ);
        }
    }
    C* N3 = (C*)g.N3;
    for (int i = 0; i < 3; ++i) {
        inverse3(3 + 3 * i, 4 + 3 * i, 5 + 3 * i, 1, i);
        // N_i = u d_x u_i + v d_y u_i + w d_z u_i, in this order, over the d_x slot
        C* G0 = Sb;
        const C* G1 = Sb + SSP;
        const C* G2 = Sb + 2 * SSP;
        for (int t = tid; t < HPL * MX; t += NT) {
            const int p = t % HPL, x = t / HPL;
            const C a = G0[t], b = G1[t], c = G2[t];
            const int i0 = x * ZL + p, i1 = i0 + HPL;
            G0[t] = mk<C>(PU[i0] * a.x + PV[i0] * b.x + PW[i0] * c.x, PU[i1] * a.y + PV[i1] * b.y + PW[i1] * c.y);
        }
        __syncthreads();
        forward(N3 + (size_t)i * fs + off0);
    }
    // no rank may leave while a peer can still write into its shared memory
    cluster.sync();
}

template <typename T, int MX, int MZ, int CL>
void launch_t(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
    typedef Cfg<T, MX, MZ, CL> K;
    k_plane_cl<T, MX, MZ, CL><<<dim3(g.ny * CL, g.E), K::NT, K::BYTES, st>>>(g, U, W);
}

template <typename T, int MX, int MZ, int CL>
void set_attr_t() {
    typedef Cfg<T, MX, MZ, CL> K;
    static_assert(K::BYTES <= 227 * 1024, "plane stage does not fit in shared memory");
    allow_max_dynamic_smem(k_plane_cl<T, MX, MZ, CL>);
}

}  // namespace pcl

// Variants in the library: (precision, Mx, Mz, cluster size)
#define DNS_PLANE_CL(X) \
    X(float, 64, 64, 2) X(float, 128, 128, 4) X(float, 128, 64, 4) X(float, 64, 128, 4) \
    X(double, 128, 128, 8) X(double, 128, 64, 8) X(double, 64, 128, 8)

bool launch_plane_cl(const GroupView& g, bool fp64, const double* U, const double* W, cudaStream_t st) {
#define DNS_CASE(T, a, b, c) \
    if ((sizeof(T) == 8) == fp64 && g.mx == a && g.mz == b) { pcl::launch_t<T, a, b, c>(g, U, W, st); return true; }
    DNS_PLANE_CL(DNS_CASE)
#undef DNS_CASE
    return false;
}

size_t plane_cl_smem_bytes(int mx, int mz, bool fp64) {
#define DNS_CASE(T, a, b, c) \
    if ((sizeof(T) == 8) == fp64 && mx == a && mz == b) return pcl::Cfg<T, a, b, c>::BYTES;
    DNS_PLANE_CL(DNS_CASE)
#undef DNS_CASE
    return 0;
}

void set_attributes_plane_cl() {
#define DNS_CASE(T, a, b, c) pcl::set_attr_t<T, a, b, c>();
    DNS_PLANE_CL(DNS_CASE)
#undef DNS_CASE
}

}  // namespace dnsk
