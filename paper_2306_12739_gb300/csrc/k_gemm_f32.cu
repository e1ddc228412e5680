// Single-precision y-contractions of the mixed path, register-tiled (each
// thread owns a 4-row x 1-complex-column micro-tile; operators are stored
// transposed and row-padded, [k][r] with r padded to RP = 4 ceil(Ny/4), so one
// 16-byte shared load feeds four rows).
//   k_yderiv_t  Dv, D2v, D eta with the shared Chebyshev operators (Sec. 3.1),
//               H layout in, P layout out
//   k_forcing_t F = -k^2 Nv - D1 (i kx Nu + i kz Nw), G = i kz Nu - i kx Nw
//               (Eqs. Dv, eta) and the RK3 combination, P layout in, H out
//   k_helm_t    x_s = x_t + (M_h - I) x_t + P_h F~ per wavenumber pair
//               (increment form of Eqs. CN1, CN2); the pair's operators arrive
//               by one TMA bulk copy (cp.async.bulk + mbarrier) per CTA.
#include "dns_internal.hpp"
#include "mbar.cuh"
#include "cvt.cuh"
#include "ff.cuh"
#include "mean.cuh"
#include "tile.cuh"

namespace dnsk {

namespace gt {

constexpr int THREADS = 256;

// --------------------------------------------------------------- y-derivs

// Tile of the y-derivative kernel: tile_of's, with fewer columns while the
// shared memory would pass YD_SMEM_MAX; the residual of D2 is staged in shared
// memory when it fits beside the tile, else read from global memory (L1).
constexpr size_t YD_SMEM_MAX = 200 * 1024;
__host__ __device__ inline size_t yd_bytes(int ny, int rp, int nc, bool stage_d2l) {
    return ((size_t)(stage_d2l ? 3 : 2) * ny * rp + 3 * (size_t)ny * 2 * nc) * sizeof(float);
}
__host__ __device__ inline Tile yd_tile(int E, int ny, int rp, int nm, int cap0) {
    Tile t = tile_of(E, ny, nm, cap0);
    while (yd_bytes(ny, rp, t.NC, false) > YD_SMEM_MAX && t.NC > 4) {
        if (t.QT > 1) t.QT /= 2;
        else t.EBT = (t.EBT + 1) / 2;
        t.NC = t.QT * t.EBT;
    }
    return t;
}
__host__ __device__ inline bool yd_stage_d2l(int ny, int rp, int nc) { return yd_bytes(ny, rp, nc, true) <= YD_SMEM_MAX; }

__global__ void __launch_bounds__(THREADS) k_yderiv_t(GroupView g, const double2* __restrict__ V,
                                                     const double2* __restrict__ H, int sprev) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, RP = g.rp, E = g.E, NM = g.nmodes;
    const Tile T = yd_tile(E, Ny, RP, NM, g.yd_cap);
    const bool stage_d2l = yd_stage_d2l(Ny, RP, T.NC);
    if (mean_finish_rows(g, sprev, (E + T.EBT - 1) / T.EBT, sm)) return;
    const int q0 = blockIdx.x * T.QT, e0 = blockIdx.y * T.EBT;
    const int NCR = 2 * T.NC;                       // real columns
    float* D1 = (float*)sm;                         // [Ny][RP]
    float* D2 = D1 + Ny * RP;
    float* D2ls = D2 + Ny * RP;                     // residual of D2 (compensated D2 v)
    float* Xv = D2ls + (stage_d2l ? Ny * RP : 0);   // [Ny][NCR], column = 2 (el QT + qq) + c
    float* Xvl = Xv + Ny * NCR;                     // residual of v: v - (double) Xv
    float* Xe = Xvl + Ny * NCR;
    {
        const float4* s1 = (const float4*)g.D1T;
        const float4* s2 = (const float4*)g.D2T;
        const float4* s3 = (const float4*)g.D2Tl;
        for (int i = threadIdx.x; i < Ny * RP / 4; i += THREADS) {
            ((float4*)D1)[i] = s1[i];
            ((float4*)D2)[i] = s2[i];
            if (stage_d2l) ((float4*)D2ls)[i] = s3[i];
        }
        // state tile, read in H order [q][y][e], written [y][(el QT + qq)]
        const int per_q = Ny * T.EBT;
        const FastDiv dPQ((unsigned)per_q), dEB((unsigned)T.EBT);
        for (int i = threadIdx.x; i < T.QT * per_q; i += THREADS) {
            const int qq = (int)dPQ.div((unsigned)i), r = i - qq * per_q;
            const int k = (int)dEB.div((unsigned)r), el = r - k * T.EBT;
            const int q = q0 + qq, e = e0 + el;
            double2 a = make_double2(0.0, 0.0), b = a;
            if (q < NM && e < E && DNS_CK(g.status, k < Ny, CK_YDERIV_T, i)) {
                const size_t o = ((size_t)q * Ny + k) * E + e;
                a = V[o];
                b = H[o];
            }
            const int c = 2 * (el * T.QT + qq);
            const float2 ah = make_float2((float)a.x, (float)a.y);
            *(float2*)&Xv[k * NCR + c] = ah;
            *(float2*)&Xvl[k * NCR + c] = make_float2((float)(a.x - (double)ah.x), (float)(a.y - (double)ah.y));
            *(float2*)&Xe[k * NCR + c] = make_float2((float)b.x, (float)b.y);
        }
    }
    __syncthreads();
    const size_t fs = (size_t)Ny * E * NM;
    float2* P = (float2*)g.P5;
    const int RB = RP / 4;
    const float* D2l = stage_d2l ? D2ls : g.D2Tl;
    const FastDiv dNC((unsigned)T.NC), dQT((unsigned)T.QT);
    for (int m = threadIdx.x; m < RB * T.NC; m += THREADS) {
        const int rb = (int)dNC.div((unsigned)m), j = m - rb * T.NC;   // consecutive threads: consecutive q
        const int r0 = 4 * rb;
        float4 av[2] = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};   // D1 v: re, im
        float bh[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};         // D2 v, float-float
        float bl[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        float4 ae[2] = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};   // D1 eta
#pragma unroll 2
        for (int k = 0; k < Ny; ++k) {
            const float4 d1 = *(const float4*)&D1[k * RP + r0];
            const float4 d2 = *(const float4*)&D2[k * RP + r0];
            const float4 d2r = *(const float4*)&D2l[k * RP + r0];
            const float2 x = *(const float2*)&Xv[k * NCR + 2 * j];
            const float2 xl = *(const float2*)&Xvl[k * NCR + 2 * j];
            const float2 h = *(const float2*)&Xe[k * NCR + 2 * j];
            av[0].x += d1.x * x.x; av[0].y += d1.y * x.x; av[0].z += d1.z * x.x; av[0].w += d1.w * x.x;
            av[1].x += d1.x * x.y; av[1].y += d1.y * x.y; av[1].z += d1.z * x.y; av[1].w += d1.w * x.y;
            // D2 v: the collocation D2 has entries up to ~N^4 / 10 that cancel in every
            // row, so a single-precision sum would lose ~1e-5 of |D2 v|: D2 and v
            // are held as single-precision pairs and the sum is compensated
            const float dh[4] = {d2.x, d2.y, d2.z, d2.w}, dl[4] = {d2r.x, d2r.y, d2r.z, d2r.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ff_add_prod2(bh[0][i], bl[0][i], dh[i], x.x, dl[i], xl.x);
                ff_add_prod2(bh[1][i], bl[1][i], dh[i], x.y, dl[i], xl.y);
            }
            ae[0].x += d1.x * h.x; ae[0].y += d1.y * h.x; ae[0].z += d1.z * h.x; ae[0].w += d1.w * h.x;
            ae[1].x += d1.x * h.y; ae[1].y += d1.y * h.y; ae[1].z += d1.z * h.y; ae[1].w += d1.w * h.y;
        }
        const int el = (int)dQT.div((unsigned)j), qq = j - el * T.QT;
        const int q = q0 + qq, e = e0 + el;
        if (q >= NM || e >= E) continue;
        const float r_av[2][4] = {{av[0].x, av[0].y, av[0].z, av[0].w}, {av[1].x, av[1].y, av[1].z, av[1].w}};
        float r_bv[2][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            r_bv[0][i] = __fadd_rn(bh[0][i], bl[0][i]);
            r_bv[1][i] = __fadd_rn(bh[1][i], bl[1][i]);
        }
        const float r_ae[2][4] = {{ae[0].x, ae[0].y, ae[0].z, ae[0].w}, {ae[1].x, ae[1].y, ae[1].z, ae[1].w}};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int y = r0 + i;
            if (y >= Ny) break;
            if (!DNS_CK(g.status, q < NM && e < E && 2 * j + 1 < NCR, CK_YDERIV_T, q)) continue;
            const size_t o = ((size_t)y * E + e) * NM + q;
            P[o] = *(const float2*)&Xv[y * NCR + 2 * j];
            P[fs + o] = make_float2(r_av[0][i], r_av[1][i]);
            P[2 * fs + o] = make_float2(r_bv[0][i], r_bv[1][i]);
            P[3 * fs + o] = *(const float2*)&Xe[y * NCR + 2 * j];
            P[4 * fs + o] = make_float2(r_ae[0][i], r_ae[1][i]);
        }
    }
}

// ---------------------------------------------------------------- forcing

__global__ void __launch_bounds__(THREADS) k_forcing_t(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, RP = g.rp, E = g.E, NM = g.nmodes, NKX = g.nkx;
    const Tile T = tile_of(E, Ny, NM);
    const FastDiv dNKX((unsigned)NKX);
    const int q0 = blockIdx.x * T.QT, e0 = blockIdx.y * T.EBT;
    const int NCR = 2 * T.NC;
    float* D1 = (float*)sm;              // [Ny][RP]
    float* PH = D1 + Ny * RP;            // phi    [Ny][NCR], column 2 (el QT + qq) + c
    float* GG = PH + Ny * NCR;           // G      [Ny][NCR]
    float* KV = GG + Ny * NCR;           // -k^2 Nv [Ny][NCR]
    const size_t fs = (size_t)Ny * E * NM;
    const float2* N3 = (const float2*)g.N3;
    {
        const float4* s1 = (const float4*)g.D1T;
        for (int i = threadIdx.x; i < Ny * RP / 4; i += THREADS) ((float4*)D1)[i] = s1[i];
        // P layout [y][e][q]: consecutive threads read consecutive q
        const int per_y = T.EBT * T.QT;
        const FastDiv dPY((unsigned)per_y), dQT((unsigned)T.QT);
        for (int i = threadIdx.x; i < Ny * per_y; i += THREADS) {
            const int k = (int)dPY.div((unsigned)i), r = i - k * per_y;
            const int el = (int)dQT.div((unsigned)r), qq = r - el * T.QT;
            const int q = q0 + qq, e = e0 + el;
            float2 ph = make_float2(0.f, 0.f), gg = ph, kv = ph;
            if (q < NM && e < E && DNS_CK(g.status, k < Ny, CK_FORCING_T, i)) {
                const size_t o = ((size_t)k * E + e) * NM + q;
                const float2 nu = N3[o], nv = N3[fs + o], nw = N3[2 * fs + o];
                const int mi = (int)dNKX.div((unsigned)q), n = q - mi * NKX;
                const float kx = g.kxtf[n], kz = g.kztf[mi];
                const float k2 = kx * kx + kz * kz;
                const float ax = kx * nu.x + kz * nw.x, ay = kx * nu.y + kz * nw.y;   // i kx Nu + i kz Nw
                ph = make_float2(-ay, ax);
                const float bx = kz * nu.x - kx * nw.x, by = kz * nu.y - kx * nw.y;   // i kz Nu - i kx Nw
                gg = make_float2(-by, bx);
                kv = make_float2(-k2 * nv.x, -k2 * nv.y);
            }
            const int c = 2 * (el * T.QT + qq);
            *(float2*)&PH[k * NCR + c] = ph;
            *(float2*)&GG[k * NCR + c] = gg;
            *(float2*)&KV[k * NCR + c] = kv;
        }
    }
    __syncthreads();
    const int RB = RP / 4;
    const FastDiv dEB2((unsigned)T.EBT), dQT2((unsigned)T.QT);
    const int q_mean = mean_mode(g);
    for (int m = threadIdx.x; m < RB * T.NC; m += THREADS) {
        // consecutive threads: consecutive members (the H layout's fastest index)
        const int r = (int)dEB2.div((unsigned)m), el = m - r * T.EBT;
        const int rb = (int)dQT2.div((unsigned)r), qq = r - rb * T.QT;
        const int j = el * T.QT + qq;
        const int r0 = 4 * rb;
        float4 ax = make_float4(0, 0, 0, 0), ay = ax;
#pragma unroll 4
        for (int k = 0; k < Ny; ++k) {
            const float4 d = *(const float4*)&D1[k * RP + r0];
            const float2 p = *(const float2*)&PH[k * NCR + 2 * j];
            ax.x += d.x * p.x; ax.y += d.y * p.x; ax.z += d.z * p.x; ax.w += d.w * p.x;
            ay.x += d.x * p.y; ay.y += d.y * p.y; ay.z += d.z * p.y; ay.w += d.w * p.y;
        }
        const int q = q0 + qq, e = e0 + el;
        if (q >= NM || e >= E) continue;
        const float rx[4] = {ax.x, ax.y, ax.z, ax.w}, ry[4] = {ay.x, ay.y, ay.z, ay.w};
        // stochastic forcing of the step in this mode's column
        const int fmi = g.fn > 0 ? q / g.nkx : 0;
        const bool forced = g.fn > 0 && q - fmi * g.nkx == g.fn;
        // RK accumulators of the four rows loaded before any store
        float2* Av = (float2*)g.Av;
        float2* Ae = (float2*)g.Ae;
        float2 pav[4], pae[4];
        if (s != 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int y = r0 + i;
                if (y >= Ny) break;
                const size_t h = ((size_t)q * Ny + y) * E + e;
                pav[i] = Av[h];
                pae[i] = Ae[h];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int y = r0 + i;
            if (y >= Ny) break;
            const float2 kv = *(const float2*)&KV[y * NCR + 2 * j];
            const float2 gg = *(const float2*)&GG[y * NCR + 2 * j];
            // F~, G~ and their RK3 accumulators in single precision: they carry the
            // accuracy of the single-precision nonlinear terms; the state itself is
            // accumulated in double by the implicit apply
            float2 F = make_float2(kv.x - rx[i], kv.y - ry[i]);
            float2 G = gg;
            if (q == q_mean) { F = make_float2(0.f, 0.f); G = F; }
            if (forced) {
                const size_t o = ((size_t)fmi * Ny + y) * E + e, half = (size_t)g.nkz * Ny * E;
                F.x += (float)g.noise[o].x; F.y += (float)g.noise[o].y;
                G.x += (float)g.noise[half + o].x; G.y += (float)g.noise[half + o].y;
            }
            const size_t h = ((size_t)q * Ny + y) * E + e;
            float2 Ft, Gt;
            if (s == 0) {
                Ft = F; Gt = G;
                Av[h] = F; Ae[h] = G;
            } else if (s == 1) {
                const float2 a = pav[i], b = pae[i];
                Ft = make_float2(2.f * F.x - a.x, 2.f * F.y - a.y);
                Gt = make_float2(2.f * G.x - b.x, 2.f * G.y - b.y);
                Av[h] = make_float2((1.f / 6.f) * a.x + (4.f / 6.f) * F.x, (1.f / 6.f) * a.y + (4.f / 6.f) * F.y);
                Ae[h] = make_float2((1.f / 6.f) * b.x + (4.f / 6.f) * G.x, (1.f / 6.f) * b.y + (4.f / 6.f) * G.y);
            } else {
                const float2 a = pav[i], b = pae[i];
                Ft = make_float2(a.x + (1.f / 6.f) * F.x, a.y + (1.f / 6.f) * F.y);
                Gt = make_float2(b.x + (1.f / 6.f) * G.x, b.y + (1.f / 6.f) * G.y);
            }
            ((float2*)g.Fv)[h] = Ft;
            ((float2*)g.Fe)[h] = Gt;
        }
    }
}

// ------------------------------------------------------------------- helm

// x_t (single precision, needM only) and F~ of the item's modes and members
// into shared memory, [Ny][NC]
__device__ __forceinline__ void helm_stage(const GroupView& g, const HelmItem& it, bool needM, float* Xs, float* Fs) {
    const int Ny = g.ny, E = g.E, ec = it.ec, NC = it.NC;
    const double2* X = it.f == 0 ? g.v_t : g.e_t;
    const float* F = (const float*)(it.f == 0 ? g.Fv : g.Fe);   // single-precision F~ (mixed path)
    const int per = Ny * 2 * ec, total = it.nq * per;
    const FastDiv dPER((unsigned)per), d2E((unsigned)(2 * ec));
    // a thread's elements in batches of four: all global loads first, then the
    // conversions and the shared stores
    constexpr int B = 4;
    for (int i0 = threadIdx.x; i0 < total; i0 += B * THREADS) {
        double xv[B];
        float fv[B];
        int so[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int i = i0 + u * THREADS;
            so[u] = -1;
            if (i >= total) continue;
            const int which = (int)dPER.div((unsigned)i), r = i - which * per;
            const int k = (int)d2E.div((unsigned)r), c = r - k * (2 * ec);
            const int q = which == 0 ? it.q1 : it.q2;
            if (!DNS_CK(g.status, q < g.nmodes && k < Ny && it.e0 + c / 2 < E, CK_HELM_T, i)) continue;
            const size_t o = ((size_t)q * Ny + k) * 2 * E + 2 * it.e0 + c;
            so[u] = k * NC + which * 2 * ec + c;
            xv[u] = needM ? ((const double*)X)[o] : 0.0;
            fv[u] = F[o];
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (so[u] < 0) continue;
            if (needM) Xs[so[u]] = d2f(xv[u]);
            Fs[so[u]] = fv[u];
        }
    }
}

// products with the transposed operators MT = (M - I)^T, PT = P^T and the
// update x+ = x_t + ((M - I) x_t + P F~) of the item's columns
__device__ __forceinline__ void helm_compute(const GroupView& g, int s, const HelmItem& it, const float* MT,
                                             const float* PT, const float* Xs, const float* Fs) {
    const int Ny = g.ny, RP = g.rp, E = g.E, NC = it.NC, ec = it.ec;
    const bool needM = (s != 2);
    const double2* X = it.f == 0 ? g.v_t : g.e_t;
    double2* M1 = it.f == 0 ? g.mx1_v : g.mx1_e;
    double2* O = (s == 2) ? (it.f == 0 ? g.v_t : g.e_t) : (it.f == 0 ? g.v_s : g.e_s);
    const int RB = RP / 4, CB = NC / 2;
    const FastDiv dCB((unsigned)CB), d2E((unsigned)(2 * ec));
    for (int m = threadIdx.x; m < RB * CB; m += THREADS) {
        const int rb = (int)dCB.div((unsigned)m), cb = m - rb * CB;
        const int r0 = 4 * rb, c0 = 2 * cb;
        float4 pa = make_float4(0, 0, 0, 0), pb = pa, ma = pa, mb = pa;   // columns c0, c0+1
#pragma unroll 4
        for (int k = 0; k < Ny; ++k) {
            const float4 pk = *(const float4*)&PT[k * RP + r0];
            const float2 fk = *(const float2*)&Fs[k * NC + c0];
            pa.x += pk.x * fk.x; pa.y += pk.y * fk.x; pa.z += pk.z * fk.x; pa.w += pk.w * fk.x;
            pb.x += pk.x * fk.y; pb.y += pk.y * fk.y; pb.z += pk.z * fk.y; pb.w += pk.w * fk.y;
            if (needM) {
                const float4 mk = *(const float4*)&MT[k * RP + r0];
                const float2 xk = *(const float2*)&Xs[k * NC + c0];
                ma.x += mk.x * xk.x; ma.y += mk.y * xk.x; ma.z += mk.z * xk.x; ma.w += mk.w * xk.x;
                mb.x += mk.x * xk.y; mb.y += mk.y * xk.y; mb.z += mk.z * xk.y; mb.w += mk.w * xk.y;
            }
        }
        const int which = (int)d2E.div((unsigned)c0), cl = 2 * it.e0 + c0 - which * 2 * ec;
        const int q = which == 0 ? it.q1 : it.q2;
        const float rp[2][4] = {{pa.x, pa.y, pa.z, pa.w}, {pb.x, pb.y, pb.z, pb.w}};
        const float rm[2][4] = {{ma.x, ma.y, ma.z, ma.w}, {mb.x, mb.y, mb.z, mb.w}};
        // x+ = x_t + ((M - I) x_t + P F~): the increment in single precision, one
        // double add; (M_1 - I) x_t of sub-step 2 is kept (single precision) for
        // sub-step 3.  In sub-step 3 the output overwrites x_t element by element.
        const double* xg = (const double*)(X + (size_t)q * Ny * E);
        float* m1 = (float*)(M1 + (size_t)q * Ny * E);
        double* og = (double*)(O + (size_t)q * Ny * E);
        // all loads of the four rows first, then the stores (the output may be
        // x_t itself, which would otherwise serialise the loads)
        double x0[4], x1[4];
        float d0[4], d1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int y = r0 + i;
            if (y >= Ny) break;
            const int o = y * 2 * E + cl;
            x0[i] = xg[o];
            x1[i] = xg[o + 1];
            if (needM) {
                d0[i] = rm[0][i];
                d1[i] = rm[1][i];
            } else {
                d0[i] = m1[o];
                d1[i] = m1[o + 1];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int y = r0 + i;
            if (y >= Ny) break;
            const int o = y * 2 * E + cl;
            if (s == 1) { m1[o] = d0[i]; m1[o + 1] = d1[i]; }
            og[o] = x0[i] + f2d(d0[i] + rp[0][i]);
            og[o + 1] = x1[i] + f2d(d1[i] + rp[1][i]);
        }
    }
}

// TMA bulk copy of the item's operators ((M - I)^T then P^T, contiguous; only
// P^T when M is not needed) into dst, completing on mbarrier bar
__device__ __forceinline__ void helm_issue(const GroupView& g, int s, const HelmItem& it, float* dst, unsigned bar) {
    const size_t mat = (size_t)g.ny * g.rp;
    const bool needM = (s != 2);
    const float* src = g.opsfT[s == 0 ? 0 : 1] + ((size_t)it.p * 4 + 2 * it.f) * mat;
    const unsigned bytes = (unsigned)((needM ? 2 : 1) * mat * sizeof(float));
    const float* from = needM ? src : src + mat;
    float* to = needM ? dst : dst + mat;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(to)), "l"(from), "r"(bytes), "r"(bar) : "memory");
}

// one CTA per (pair, field, member chunk)
__global__ void __launch_bounds__(THREADS, 3) k_helm_t(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, RP = g.rp, E = g.E, NKX = g.nkx;
    // leading CTAs: rows of the mean-flow update (independent work that fills
    // SMs beside the wavenumber pairs), finished by launch_mean_finish
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_rows(g, s, blockIdx.x % E, (blockIdx.x / E) * (THREADS / 32), sm);
        return;
    }
    const int b = blockIdx.x - nrow;
    const int p = b % g.npairs, f = (b / g.npairs) & 1, ch = b / (2 * g.npairs);
    if (!g.lin && p % NKX == 0 && p / NKX == 0) return;   // the mean mode (DNS groups)
    const HelmItem it = helm_item(g, p, f, ch);
    const size_t mat = (size_t)Ny * RP;           // floats per transposed operator
    float* MT = (float*)sm;                       // [Ny][RP]  (M - I)^T
    float* PT = MT + mat;                         // [Ny][RP]  P^T
    float* Xs = PT + mat;                         // [Ny][NC]
    float* Fs = Xs + (size_t)Ny * it.NC;          // [Ny][NC]
    unsigned long long* bar = (unsigned long long*)(Fs + (size_t)Ny * it.NC + 2);
    const unsigned bar_a = su32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) helm_issue(g, s, it, MT, bar_a);
    helm_stage(g, it, s != 2, Xs, Fs);
    __syncthreads();
    if (!mbar_wait(bar_a, 0)) {
        // the operator copy did not land: flag it, give the copy one more bounded
        // wait so no write into this CTA's shared memory is left in flight, leave
        if (threadIdx.x == 0) atomicExch(g.status, 1);
        mbar_wait(bar_a, 0);
        return;
    }
    helm_compute(g, s, it, MT, PT, Xs, Fs);
}

// Persistent variant: after the mean-row CTAs, every CTA loops over work items
// (the valid (pair, field, chunk) triples, the DNS mean mode left out) with the
// grid stride, and while it computes one item the TMA copy of its next item's
// operators lands in the other of two buffers.  Every thread takes part in
// every bounded wait and the CTA decides together (__syncthreads_and), so a
// wait that gives up ends the whole CTA, after one more bounded wait for each
// copy still in flight.
__global__ void __launch_bounds__(THREADS, 3) k_helm_tp(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, RP = g.rp, E = g.E;
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_rows(g, s, blockIdx.x % E, (blockIdx.x / E) * (THREADS / 32), sm);
        return;
    }
    const int npv = g.lin ? g.npairs : g.npairs - 1, p0 = g.lin ? 0 : 1;
    const int nitems = 2 * npv * helm_member_chunks(g);
    const int stride = gridDim.x - nrow;
    const size_t mat = (size_t)Ny * RP;
    float* OP0 = (float*)sm;                      // [2][Ny][RP] (M - I)^T, P^T
    float* OP1 = OP0 + 2 * mat;
    float* Xs = OP1 + 2 * mat;
    float* Fs = Xs + (size_t)Ny * 4 * helm_member_chunk(g);
    unsigned long long* bars = (unsigned long long*)(Fs + (size_t)Ny * 4 * helm_member_chunk(g) + 2);
    const unsigned bar0 = su32(bars), bar1 = su32(bars + 1);
    auto decode = [&](int t) {
        const int p = p0 + t % npv, f = (t / npv) & 1, ch = t / (2 * npv);
        return helm_item(g, p, f, ch);
    };
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int t = blockIdx.x - nrow;
    if (t < nitems && threadIdx.x == 0) helm_issue(g, s, decode(t), OP0, bar0);
    unsigned ph0 = 0, ph1 = 0;
    for (int buf = 0; t < nitems; t += stride, buf ^= 1) {
        const HelmItem it = decode(t);
        helm_stage(g, it, s != 2, Xs, Fs);
        // staging done, and every thread finished the previous item (whose
        // operator buffer the next copy reuses)
        __syncthreads();
        const int tn = t + stride;
        if (tn < nitems && threadIdx.x == 0) helm_issue(g, s, decode(tn), buf ? OP0 : OP1, buf ? bar0 : bar1);
        const bool ok = mbar_wait(buf ? bar1 : bar0, buf ? ph1 : ph0);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicExch(g.status, 1);
                mbar_wait(buf ? bar1 : bar0, buf ? ph1 : ph0);
                if (tn < nitems) mbar_wait(buf ? bar0 : bar1, buf ? ph0 : ph1);
            }
            return;
        }
        if (buf) ph1 ^= 1u; else ph0 ^= 1u;
        const float* OP = buf ? OP1 : OP0;
        helm_compute(g, s, it, OP, OP + mat, Xs, Fs);
        __syncthreads();   // Xs, Fs are restaged for the next item
    }
}

// Self-test of the bounded-wait path: an mbarrier that expects one arrival that
// never comes.  The wait gives up after its iteration limit and latches status.
__global__ void k_wait_selftest(int* status) {
    __shared__ unsigned long long bar;
    const unsigned b = su32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!mbar_wait(b, 0) && threadIdx.x == 0) atomicExch(status, 2);
}

}  // namespace gt

void launch_wait_selftest(int* status, cudaStream_t st) { gt::k_wait_selftest<<<1, 32, 0, st>>>(status); }

// Self-test of the bounds-check reporting: one check whose condition is false
// (index 12345 against a limit of 0), touching no memory; recorded only by the
// checked build.
__global__ void k_bounds_selftest(int* status) {
    const long long idx = 12345 + threadIdx.x;
    (void)DNS_CK(status, idx < 0, CK_SELFTEST, idx);
}
void launch_bounds_selftest(int* status, cudaStream_t st) { k_bounds_selftest<<<1, 1, 0, st>>>(status); }

size_t helm_t_smem_bytes(const GroupView& g) {
    const int nc = 2 * 2 * helm_member_chunk(g);
    size_t b = (2 * (size_t)g.ny * g.rp + 2 * (size_t)g.ny * nc + 2) * sizeof(float) + 16;
    size_t m = mean_smem_bytes(g);
    return b > m ? b : m;
}

size_t yderiv_t_smem_bytes(const GroupView& g) {
    gt::Tile t = gt::yd_tile(g.E, g.ny, g.rp, g.nmodes, g.yd_cap);
    return gt::yd_bytes(g.ny, g.rp, t.NC, gt::yd_stage_d2l(g.ny, g.rp, t.NC));
}

size_t forcing_t_smem_bytes(const GroupView& g) {
    gt::Tile t = gt::tile_of(g.E, g.ny, g.nmodes);
    return ((size_t)g.ny * g.rp + 3 * (size_t)g.ny * 2 * t.NC) * sizeof(float);
}

void launch_yderiv_t(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev) {
    gt::Tile t = gt::yd_tile(g.E, g.ny, g.rp, g.nmodes, g.yd_cap);
    dim3 grid((g.nmodes + t.QT - 1) / t.QT, (g.E + t.EBT - 1) / t.EBT);
    grid.y += mean_finish_extra_rows(g, grid.x, sprev);
    gt::k_yderiv_t<<<grid, gt::THREADS, yderiv_t_smem_bytes(g), st>>>(g, v, e, sprev);
}

void launch_forcing_t(const GroupView& g, int s, cudaStream_t st) {
    gt::Tile t = gt::tile_of(g.E, g.ny, g.nmodes);
    dim3 grid((g.nmodes + t.QT - 1) / t.QT, (g.E + t.EBT - 1) / t.EBT);
    gt::k_forcing_t<<<grid, gt::THREADS, forcing_t_smem_bytes(g), st>>>(g, s);
}

void launch_helm_t(const GroupView& g, int s, cudaStream_t st) {
    gt::k_helm_t<<<mean_row_ctas(g) + 2 * g.npairs * helm_member_chunks(g), gt::THREADS, helm_t_smem_bytes(g), st>>>(
        g, s);
}

size_t helm_tp_smem_bytes(const GroupView& g) {
    const int nc = 2 * 2 * helm_member_chunk(g);
    size_t b = (4 * (size_t)g.ny * g.rp + 2 * (size_t)g.ny * nc + 2) * sizeof(float) + 2 * 8 + 16;
    size_t m = mean_smem_bytes(g);
    return b > m ? b : m;
}

// persistent CTAs: as many as fit on the GPU at once (never more than items)
void launch_helm_tp(const GroupView& g, int s, cudaStream_t st) {
    static int n_sm = 0, occ = 0;
    static size_t occ_smem = 0;
    const size_t smem = helm_tp_smem_bytes(g);
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    if (occ_smem != smem) {
        occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gt::k_helm_tp, gt::THREADS, smem);
        if (occ < 1) occ = 1;
        occ_smem = smem;
    }
    const int nitems = 2 * (g.lin ? g.npairs : g.npairs - 1) * helm_member_chunks(g);
    int np = occ * (n_sm > 0 ? n_sm : 1);
    if (np > nitems) np = nitems;
    if (np < 1) np = 1;
    gt::k_helm_tp<<<mean_row_ctas(g) + np, gt::THREADS, smem, st>>>(g, s);
}

void set_attributes_gemm_t() {
    allow_max_dynamic_smem(gt::k_yderiv_t);
    allow_max_dynamic_smem(gt::k_forcing_t);
    allow_max_dynamic_smem(gt::k_helm_t);
    allow_max_dynamic_smem(gt::k_helm_tp);
}

}  // namespace dnsk
