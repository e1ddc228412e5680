// The step-by-step per-wavenumber stage of the mixed path in parity blocks
// (eo.cuh): the y-derivatives (Dv, D2v, D eta, Sec. 3.1), the forcing (Eqs.
// Dv, eta: D1 phi) and the implicit apply (increment form of Eqs. CN1, CN2:
// (M - I) x_t + P F~), each product as the even and odd halves of its
// operator, half the operator bytes and multiply-adds of the natural-order
// kernels (k_gemm_f32.cu: k_yderiv_t, k_forcing_t, k_helm_t), whose tiles,
// work items and epilogues these follow.  The state,
// forcings and accumulators stay in the natural order in global memory; the
// staging converts the two natural rows of each pair-row into parity parts and
// every task converts its products back.
#include "dns_internal.hpp"
#include "mbar.cuh"
#include "cvt.cuh"
#include "ff.cuh"
#include "mean.cuh"
#include "tile.cuh"
#include "eo.cuh"

namespace dnsk {

namespace sto {

using spc::eo2;
using spc::eo2x2;
using spc::eo_rows;
using spc::EoRows;

constexpr int THREADS = 256;

// ----------------------------------------------------------- y-derivatives

// Column tile of the y-derivatives in parity blocks: tile_of's, with fewer
// columns while the shared memory (D1, D2 and its residual in parity blocks,
// three vectors) would pass YDE_SMEM_MAX.
constexpr size_t YDE_SMEM_MAX = 200 * 1024;
__host__ __device__ inline size_t yde_bytes(int ny, int nc) {
    return (3 * spc::eo_mat(ny) + 3 * (size_t)ny * 2 * nc) * sizeof(float);
}
__host__ __device__ inline gt::Tile yde_tile(int E, int ny, int nm, int cap0) {
    gt::Tile t = gt::tile_of(E, ny, nm, cap0);
    while (yde_bytes(ny, t.NC) > YDE_SMEM_MAX && t.NC > 4) {
        if (t.QT > 1) t.QT /= 2;
        else t.EBT = (t.EBT + 1) / 2;
        t.NC = t.QT * t.EBT;
    }
    return t;
}

// Dv, D2v, D eta of a column tile (k_yderiv_t's tile and output): v staged as
// the float-float even and odd parts of the FP64 state, eta as single-precision
// sums; D1 (anti-centro-symmetric) maps the odd part to the even output rows
// and the even part to the odd ones, D2 (centro-symmetric, float-float with its
// residual) maps each part to its own.  Tasks: two pair-rows x one complex
// column.  Grid rows from (E + EBT - 1) / EBT on finish the previous sub-step's
// mean flow (one CTA per member).
__global__ void __launch_bounds__(THREADS) k_yderiv_eo(GroupView g, const double2* __restrict__ V,
                                                      const double2* __restrict__ H, int sprev) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, E = g.E, NM = g.nmodes;
    const gt::Tile T = yde_tile(E, Ny, NM, g.yd_cap);
    if (mean_finish_rows(g, sprev, (E + T.EBT - 1) / T.EBT, sm)) return;
    const int NE = (Ny + 1) / 2, NO = Ny / 2, RP2 = spc::eo_rp(Ny), RB2 = (NE + 1) / 2;
    const size_t MEO = spc::eo_mat(Ny);
    const int q0 = blockIdx.x * T.QT, e0 = blockIdx.y * T.EBT;
    const int NCR = 2 * T.NC;
    float* D1 = (float*)sm;                       // D1 in parity blocks
    float* D2 = D1 + MEO;                         // D2
    float* D2l = D2 + MEO;                        // its residual
    float* Xh = D2l + MEO;                        // v parts, high [Ny][NCR]
    float* Xl = Xh + (size_t)Ny * NCR;            // v parts, low
    float* Xe = Xl + (size_t)Ny * NCR;            // eta parts
    const size_t fs = (size_t)Ny * E * NM;
    float2* P = (float2*)g.P5;
    {
        const float4* s1 = (const float4*)g.D1EO;
        const float4* s2 = (const float4*)g.D2EO;
        const float4* s3 = (const float4*)g.D2lEO;
        for (int i = threadIdx.x; i < (int)(MEO / 4); i += THREADS) {
            ((float4*)D1)[i] = s1[i];
            ((float4*)D2)[i] = s2[i];
            ((float4*)D2l)[i] = s3[i];
        }
        // state tile, read in H order [q][y][e] (consecutive threads: consecutive
        // members), both natural rows of a pair-row per thread; v and eta in single
        // precision into their planes of the P layout
        const int per_q = NE * T.EBT;
        const FastDiv dPQ((unsigned)per_q), dEB((unsigned)T.EBT);
        for (int i = threadIdx.x; i < T.QT * per_q; i += THREADS) {
            const int qq = (int)dPQ.div((unsigned)i), r = i - qq * per_q;
            const int p = (int)dEB.div((unsigned)r), el = r - p * T.EBT;
            const int q = q0 + qq, e = e0 + el;
            const EoRows R = eo_rows(p, Ny);
            double2 a[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)}, b[2] = {a[0], a[1]};
            if (q < NM && e < E && DNS_CK(g.status, R.y1 < Ny, CK_YDERIV_T, i)) {
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    if (k2 && !R.pair) continue;
                    const int y = k2 ? R.y1 : R.y0;
                    const size_t oh = ((size_t)q * Ny + y) * E + e, op = ((size_t)y * E + e) * NM + q;
                    a[k2] = V[oh];
                    b[k2] = H[oh];
                    P[op] = make_float2(d2f(a[k2].x), d2f(a[k2].y));
                    P[3 * fs + op] = make_float2(d2f(b[k2].x), d2f(b[k2].y));
                }
            }
            const int c = 2 * (el * T.QT + qq);
            float2 he, le, ho, lo;
            spc::eo_ff(a[0].x, a[1].x, he.x, le.x, ho.x, lo.x);
            spc::eo_ff(a[0].y, a[1].y, he.y, le.y, ho.y, lo.y);
            const float2 h0 = make_float2(d2f(b[0].x), d2f(b[0].y)), h1 = make_float2(d2f(b[1].x), d2f(b[1].y));
            *(float2*)&Xh[p * NCR + c] = he;
            *(float2*)&Xl[p * NCR + c] = le;
            *(float2*)&Xe[p * NCR + c] = make_float2(h0.x + h1.x, h0.y + h1.y);
            if (R.pair) {
                *(float2*)&Xh[(NE + p) * NCR + c] = ho;
                *(float2*)&Xl[(NE + p) * NCR + c] = lo;
                *(float2*)&Xe[(NE + p) * NCR + c] = make_float2(h0.x - h1.x, h0.y - h1.y);
            }
        }
    }
    __syncthreads();
    const FastDiv dNC((unsigned)T.NC), dQT((unsigned)T.QT);
    // the odd-output block of D1 (after its NO even-output rows), the odd-output
    // block of D2 and its residual (after their NE even-output rows)
    const float* D1o = D1 + (size_t)NO * RP2;
    const float* D2o = D2 + (size_t)NE * RP2;
    const float* D2lo = D2l + (size_t)NE * RP2;
    for (int m = threadIdx.x; m < RB2 * T.NC; m += THREADS) {
        const int rb = (int)dNC.div((unsigned)m), j = m - rb * T.NC;   // consecutive threads: consecutive q
        const int p0 = 2 * rb, c2 = 2 * j;
        float d1o[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, f1o[2][2] = {{0.f, 0.f}, {0.f, 0.f}};   // D1 v, D1 eta: odd rows
        float d1e[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, f1e[2][2] = {{0.f, 0.f}, {0.f, 0.f}};   // even rows
        float beh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, bel[2][2] = {{0.f, 0.f}, {0.f, 0.f}};   // D2 v even rows
        float boh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, bol[2][2] = {{0.f, 0.f}, {0.f, 0.f}};   // D2 v odd rows
        // the even parts: D1's odd-output block, D2's even-output block
#pragma unroll 2
        for (int k = 0; k < NE; ++k) {
            const float2 b1 = *(const float2*)&D1o[k * RP2 + p0];
            const float2 b2 = *(const float2*)&D2[k * RP2 + p0];
            const float2 b2l = *(const float2*)&D2l[k * RP2 + p0];
            const float2 x = *(const float2*)&Xh[k * NCR + c2];
            const float2 xl = *(const float2*)&Xl[k * NCR + c2];
            const float2 h = *(const float2*)&Xe[k * NCR + c2];
            const float bb1[2] = {b1.x, b1.y}, bb2[2] = {b2.x, b2.y}, bbl[2] = {b2l.x, b2l.y};
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                d1o[r][0] += bb1[r] * x.x; d1o[r][1] += bb1[r] * x.y;
                f1o[r][0] += bb1[r] * h.x; f1o[r][1] += bb1[r] * h.y;
                ff_add_prod2(beh[r][0], bel[r][0], bb2[r], x.x, bbl[r], xl.x);
                ff_add_prod2(beh[r][1], bel[r][1], bb2[r], x.y, bbl[r], xl.y);
            }
        }
        // the odd parts: D1's even-output block, D2's odd-output block
#pragma unroll 2
        for (int k = 0; k < NO; ++k) {
            const float2 b1 = *(const float2*)&D1[k * RP2 + p0];
            const float2 b2 = *(const float2*)&D2o[k * RP2 + p0];
            const float2 b2l = *(const float2*)&D2lo[k * RP2 + p0];
            const float2 x = *(const float2*)&Xh[(NE + k) * NCR + c2];
            const float2 xl = *(const float2*)&Xl[(NE + k) * NCR + c2];
            const float2 h = *(const float2*)&Xe[(NE + k) * NCR + c2];
            const float bb1[2] = {b1.x, b1.y}, bb2[2] = {b2.x, b2.y}, bbl[2] = {b2l.x, b2l.y};
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                d1e[r][0] += bb1[r] * x.x; d1e[r][1] += bb1[r] * x.y;
                f1e[r][0] += bb1[r] * h.x; f1e[r][1] += bb1[r] * h.y;
                ff_add_prod2(boh[r][0], bol[r][0], bb2[r], x.x, bbl[r], xl.x);
                ff_add_prod2(boh[r][1], bol[r][1], bb2[r], x.y, bbl[r], xl.y);
            }
        }
        const int el = (int)dQT.div((unsigned)j), qq = j - el * T.QT;
        const int q = q0 + qq, e = e0 + el;
        if (q >= NM || e >= E) continue;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int p = p0 + r;
            if (p >= NE) break;
            const EoRows R = eo_rows(p, Ny);
            const float ve[2] = {__fadd_rn(beh[r][0], bel[r][0]), __fadd_rn(beh[r][1], bel[r][1])};
            const float vo[2] = {__fadd_rn(boh[r][0], bol[r][0]), __fadd_rn(boh[r][1], bol[r][1])};
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                if (k2 && !R.pair) continue;
                const int y = k2 ? R.y1 : R.y0;
                if (!DNS_CK(g.status, 2 * j + 1 < NCR, CK_YDERIV_T, q)) continue;
                const float sg = k2 ? -1.f : 1.f;
                const size_t o = ((size_t)y * E + e) * NM + q;
                P[fs + o] = R.pair ? make_float2(0.5f * (d1e[r][0] + sg * d1o[r][0]), 0.5f * (d1e[r][1] + sg * d1o[r][1]))
                                   : make_float2(d1e[r][0], d1e[r][1]);
                P[2 * fs + o] = R.pair ? make_float2(0.5f * (ve[0] + sg * vo[0]), 0.5f * (ve[1] + sg * vo[1]))
                                       : make_float2(ve[0], ve[1]);
                P[4 * fs + o] = R.pair ? make_float2(0.5f * (f1e[r][0] + sg * f1o[r][0]), 0.5f * (f1e[r][1] + sg * f1o[r][1]))
                                       : make_float2(f1e[r][0], f1e[r][1]);
            }
        }
    }
}

// ---------------------------------------------------------------- forcing

// Column tile of k_forcing_t; D1 in parity blocks, phi in parity parts, G and
// -k^2 Nv in natural rows.  Tasks: two pair-rows x one complex column.
__global__ void __launch_bounds__(THREADS) k_forcing_eo(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, E = g.E, NM = g.nmodes, NKX = g.nkx;
    const int NE = (Ny + 1) / 2, NO = Ny / 2, RP2 = spc::eo_rp(Ny), RB2 = (NE + 1) / 2;
    const size_t MEO = spc::eo_mat(Ny);
    const gt::Tile T = gt::tile_of(E, Ny, NM);
    const FastDiv dNKX((unsigned)NKX);
    const int q0 = blockIdx.x * T.QT, e0 = blockIdx.y * T.EBT;
    const int NCR = 2 * T.NC;
    float* D1 = (float*)sm;                       // D1 in parity blocks
    float* PH = D1 + MEO;                         // phi in parity parts [Ny][NCR]
    float* GG = PH + (size_t)Ny * NCR;            // G       [Ny][NCR], natural rows
    float* KV = GG + (size_t)Ny * NCR;            // -k^2 Nv [Ny][NCR], natural rows
    const size_t fs = (size_t)Ny * E * NM;
    const float2* N3 = (const float2*)g.N3;
    {
        const float4* s1 = (const float4*)g.D1EO;
        for (int i = threadIdx.x; i < (int)(MEO / 4); i += THREADS) ((float4*)D1)[i] = s1[i];
        const int per_y = T.EBT * T.QT;
        const FastDiv dPY((unsigned)per_y), dQT((unsigned)T.QT);
        for (int i = threadIdx.x; i < NE * per_y; i += THREADS) {
            const int p = (int)dPY.div((unsigned)i), r = i - p * per_y;
            const int el = (int)dQT.div((unsigned)r), qq = r - el * T.QT;
            const int q = q0 + qq, e = e0 + el;
            const EoRows R = eo_rows(p, Ny);
            const int c = 2 * (el * T.QT + qq);
            float2 ph[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                if (k2 && !R.pair) continue;
                const int y = k2 ? R.y1 : R.y0;
                float2 gg = make_float2(0.f, 0.f), kv = gg;
                if (q < NM && e < E && DNS_CK(g.status, y < Ny, CK_FORCING_T, i)) {
                    const size_t o = ((size_t)y * E + e) * NM + q;
                    const float2 nu = N3[o], nv = N3[fs + o], nw = N3[2 * fs + o];
                    const int mi = (int)dNKX.div((unsigned)q), n = q - mi * NKX;
                    const float kx = g.kxtf[n], kz = g.kztf[mi];
                    const float k2n = kx * kx + kz * kz;
                    const float ax = kx * nu.x + kz * nw.x, ay = kx * nu.y + kz * nw.y;   // i kx Nu + i kz Nw
                    ph[k2] = make_float2(-ay, ax);
                    const float bx = kz * nu.x - kx * nw.x, by = kz * nu.y - kx * nw.y;   // i kz Nu - i kx Nw
                    gg = make_float2(-by, bx);
                    kv = make_float2(-k2n * nv.x, -k2n * nv.y);
                }
                *(float2*)&GG[y * NCR + c] = gg;
                *(float2*)&KV[y * NCR + c] = kv;
            }
            *(float2*)&PH[p * NCR + c] = make_float2(ph[0].x + ph[1].x, ph[0].y + ph[1].y);
            if (R.pair) *(float2*)&PH[(NE + p) * NCR + c] = make_float2(ph[0].x - ph[1].x, ph[0].y - ph[1].y);
        }
    }
    __syncthreads();
    const FastDiv dEB2((unsigned)T.EBT), dQT2((unsigned)T.QT);
    const int q_mean = mean_mode(g);
    float2* Av = (float2*)g.Av;
    float2* Ae = (float2*)g.Ae;
    for (int m = threadIdx.x; m < RB2 * T.NC; m += THREADS) {
        // consecutive threads: consecutive members (the H layout's fastest index)
        const int r = (int)dEB2.div((unsigned)m), el = m - r * T.EBT;
        const int rb = (int)dQT2.div((unsigned)r), qq = r - rb * T.QT;
        const int j = el * T.QT + qq, p0 = 2 * rb;
        const int q = q0 + qq, e = e0 + el;
        if (q >= NM || e >= E) continue;
        // D1 phi: the even rows contract the odd part, the odd rows the even part
        float ye[2][2], yo[2][2];
        eo2(D1, NO, NE, RP2, PH + NE * NCR, PH, NCR, p0, 2 * j, ye, yo);
        const int fmi = g.fn > 0 ? q / g.nkx : 0;
        const bool forced = g.fn > 0 && q - fmi * g.nkx == g.fn;
        // the RK accumulators of the (up to four) natural rows before any store
        float2 pav[2][2], pae[2][2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                pav[rr][k2] = pae[rr][k2] = make_float2(0.f, 0.f);
                const EoRows R = eo_rows(p0 + rr, Ny);
                if (s == 0 || p0 + rr >= NE || (k2 && !R.pair)) continue;
                const size_t h = ((size_t)q * Ny + (k2 ? R.y1 : R.y0)) * E + e;
                pav[rr][k2] = Av[h];
                pae[rr][k2] = Ae[h];
            }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int p = p0 + rr;
            if (p >= NE) break;
            const EoRows R = eo_rows(p, Ny);
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                if (k2 && !R.pair) continue;
                const int y = k2 ? R.y1 : R.y0;
                const float sg = k2 ? -1.f : 1.f;
                const float dx = R.pair ? 0.5f * (ye[rr][0] + sg * yo[rr][0]) : ye[rr][0];
                const float dy = R.pair ? 0.5f * (ye[rr][1] + sg * yo[rr][1]) : ye[rr][1];
                const float2 kv = *(const float2*)&KV[y * NCR + 2 * j];
                const float2 gg = *(const float2*)&GG[y * NCR + 2 * j];
                float2 F = make_float2(kv.x - dx, kv.y - dy);
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
                    const float2 a = pav[rr][k2], b = pae[rr][k2];
                    Ft = make_float2(2.f * F.x - a.x, 2.f * F.y - a.y);
                    Gt = make_float2(2.f * G.x - b.x, 2.f * G.y - b.y);
                    Av[h] = make_float2((1.f / 6.f) * a.x + (4.f / 6.f) * F.x, (1.f / 6.f) * a.y + (4.f / 6.f) * F.y);
                    Ae[h] = make_float2((1.f / 6.f) * b.x + (4.f / 6.f) * G.x, (1.f / 6.f) * b.y + (4.f / 6.f) * G.y);
                } else {
                    const float2 a = pav[rr][k2], b = pae[rr][k2];
                    Ft = make_float2(a.x + (1.f / 6.f) * F.x, a.y + (1.f / 6.f) * F.y);
                    Gt = make_float2(b.x + (1.f / 6.f) * G.x, b.y + (1.f / 6.f) * G.y);
                }
                ((float2*)g.Fv)[h] = Ft;
                ((float2*)g.Fe)[h] = Gt;
            }
        }
    }
}

// ------------------------------------------------------------------- apply

// x_t (single precision, needM only) and F~ of the item's modes and members in
// parity parts, [Ny][NC]: rows 0..NE-1 the even part, rows NE.. the odd part;
// each part a single-precision sum of the two natural rows' values
__device__ __forceinline__ void stage_eo(const GroupView& g, const gt::HelmItem& it, bool needM, float* Xs, float* Fs) {
    const int Ny = g.ny, E = g.E, ec = it.ec, NC = it.NC, NE = (Ny + 1) / 2;
    const double* X = (const double*)(it.f == 0 ? g.v_t : g.e_t);
    const float* F = (const float*)(it.f == 0 ? g.Fv : g.Fe);
    const int per = NE * 2 * ec, total = it.nq * per;
    const FastDiv dPER((unsigned)per), d2E((unsigned)(2 * ec));
    for (int i = threadIdx.x; i < total; i += THREADS) {
        const int which = (int)dPER.div((unsigned)i), r = i - which * per;
        const int p = (int)d2E.div((unsigned)r), c = r - p * (2 * ec);
        const int q = which == 0 ? it.q1 : it.q2;
        const EoRows R = eo_rows(p, Ny);
        if (!DNS_CK(g.status, q < g.nmodes && R.y1 < Ny && it.e0 + c / 2 < E, CK_HELM_T, i)) continue;
        const size_t o0 = ((size_t)q * Ny + R.y0) * 2 * E + 2 * it.e0 + c;
        const size_t o1 = ((size_t)q * Ny + R.y1) * 2 * E + 2 * it.e0 + c;
        const double x0 = needM ? X[o0] : 0.0, x1 = (needM && R.pair) ? X[o1] : 0.0;
        const float f0 = F[o0], f1 = R.pair ? F[o1] : 0.f;
        const int col = which * 2 * ec + c;
        const float h0 = d2f(x0), h1 = d2f(x1);
        if (needM) Xs[p * NC + col] = h0 + h1;
        Fs[p * NC + col] = f0 + f1;
        if (R.pair) {
            if (needM) Xs[(NE + p) * NC + col] = h0 - h1;
            Fs[(NE + p) * NC + col] = f0 - f1;
        }
    }
}

// (M - I) x_t + P F~ of two pair-rows x one complex column per task, back in
// natural rows, and the update x+ = x_t + that increment (k_helm_t's epilogue)
__device__ __forceinline__ void compute_eo(const GroupView& g, int s, const gt::HelmItem& it, const float* MS,
                                           const float* PS, const float* Xs, const float* Fs) {
    const int Ny = g.ny, E = g.E, NC = it.NC, ec = it.ec;
    const int NE = (Ny + 1) / 2, NO = Ny / 2, RP2 = spc::eo_rp(Ny), RB2 = (NE + 1) / 2;
    const bool needM = (s != 2);
    const double2* X = it.f == 0 ? g.v_t : g.e_t;
    double2* M1 = it.f == 0 ? g.mx1_v : g.mx1_e;
    double2* O = (s == 2) ? (it.f == 0 ? g.v_t : g.e_t) : (it.f == 0 ? g.v_s : g.e_s);
    const int CB = NC / 2;
    const FastDiv dCB((unsigned)CB), d2E((unsigned)(2 * ec));
    for (int m = threadIdx.x; m < RB2 * CB; m += THREADS) {
        const int rb = (int)dCB.div((unsigned)m), cb = m - rb * CB;
        const int p0 = 2 * rb, c0 = 2 * cb;
        float ae[2][2], ao[2][2], be[2][2], bo[2][2];
        eo2x2(MS, PS, NE, NO, RP2, Xs, Xs + NE * NC, Fs, Fs + NE * NC, NC, p0, c0, needM, ae, ao, be, bo);
        const int which = (int)d2E.div((unsigned)c0), cl = 2 * it.e0 + c0 - which * 2 * ec;
        const int q = which == 0 ? it.q1 : it.q2;
        const double* xg = (const double*)(X + (size_t)q * Ny * E);
        float* m1 = (float*)(M1 + (size_t)q * Ny * E);
        double* og = (double*)(O + (size_t)q * Ny * E);
        // every load of the (up to four) rows before the stores: the output may
        // be x_t itself
        double x0[2][2], x1[2][2];
        float d0[2][2], d1[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                const int p = p0 + r;
                const EoRows R = eo_rows(p, Ny);
                x0[r][k2] = x1[r][k2] = 0.0;
                d0[r][k2] = d1[r][k2] = 0.f;
                if (p >= NE || (k2 && !R.pair)) continue;
                const int o = (k2 ? R.y1 : R.y0) * 2 * E + cl;
                x0[r][k2] = xg[o];
                x1[r][k2] = xg[o + 1];
                if (needM) {
                    const float sg = k2 ? -1.f : 1.f;
                    d0[r][k2] = R.pair ? 0.5f * (ae[r][0] + sg * ao[r][0]) : ae[r][0];
                    d1[r][k2] = R.pair ? 0.5f * (ae[r][1] + sg * ao[r][1]) : ae[r][1];
                } else {
                    d0[r][k2] = m1[o];
                    d1[r][k2] = m1[o + 1];
                }
            }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                const int p = p0 + r;
                const EoRows R = eo_rows(p, Ny);
                if (p >= NE || (k2 && !R.pair)) continue;
                const int o = (k2 ? R.y1 : R.y0) * 2 * E + cl;
                const float sg = k2 ? -1.f : 1.f;
                const float pa0 = R.pair ? 0.5f * (be[r][0] + sg * bo[r][0]) : be[r][0];
                const float pa1 = R.pair ? 0.5f * (be[r][1] + sg * bo[r][1]) : be[r][1];
                if (s == 1) { m1[o] = d0[r][k2]; m1[o + 1] = d1[r][k2]; }
                og[o] = x0[r][k2] + f2d(d0[r][k2] + pa0);
                og[o + 1] = x1[r][k2] + f2d(d1[r][k2] + pa1);
            }
    }
}

// one CTA per (pair, field, member chunk) after the mean-row CTAs, as k_helm_t;
// the item's two operators in parity blocks arrive by one TMA bulk copy
__global__ void __launch_bounds__(THREADS, 3) k_helm_eo(GroupView g, int s) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, NKX = g.nkx;
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_rows(g, s, blockIdx.x % g.E, (blockIdx.x / g.E) * (THREADS / 32), sm);
        return;
    }
    const int b = blockIdx.x - nrow;
    const int p = b % g.npairs, f = (b / g.npairs) & 1, ch = b / (2 * g.npairs);
    if (!g.lin && p % NKX == 0 && p / NKX == 0) return;   // the mean mode (DNS groups)
    const gt::HelmItem it = gt::helm_item(g, p, f, ch);
    const size_t MEO = spc::eo_mat(Ny);
    float* MS = (float*)sm;                       // M - I in parity blocks
    float* PS = MS + MEO;                         // P in parity blocks
    float* Xs = PS + MEO;                         // [Ny][NC]
    float* Fs = Xs + (size_t)Ny * it.NC;          // [Ny][NC]
    unsigned long long* bar = (unsigned long long*)(Fs + (size_t)Ny * it.NC + 2);
    const unsigned bar_a = su32(bar);
    const bool needM = (s != 2);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const float* src = g.opsEO[s == 0 ? 0 : 1] + ((size_t)p * 4 + 2 * f) * MEO;
        const unsigned bytes = (unsigned)((needM ? 2 : 1) * MEO * sizeof(float));
        const float* from = needM ? src : src + MEO;
        float* to = needM ? MS : PS;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(su32(to)), "l"(from), "r"(bytes), "r"(bar_a) : "memory");
    }
    stage_eo(g, it, needM, Xs, Fs);
    __syncthreads();
    if (!mbar_wait(bar_a, 0)) {
        // the operator copy did not land: flag it, give the copy one more bounded
        // wait so no write into this CTA's shared memory is left in flight, leave
        if (threadIdx.x == 0) atomicExch(g.status, 1);
        mbar_wait(bar_a, 0);
        return;
    }
    compute_eo(g, s, it, MS, PS, Xs, Fs);
}

}  // namespace sto

// ------------------------------------------------------------------- host

size_t forcing_eo_smem_bytes(const GroupView& g) {
    gt::Tile t = gt::tile_of(g.E, g.ny, g.nmodes);
    return (spc::eo_mat(g.ny) + 3 * (size_t)g.ny * 2 * t.NC) * sizeof(float);
}

size_t helm_eo_smem_bytes(const GroupView& g) {
    const int nc = 2 * 2 * helm_member_chunk(g);
    size_t b = (2 * spc::eo_mat(g.ny) + 2 * (size_t)g.ny * nc + 2) * sizeof(float) + 16;
    size_t m = mean_smem_bytes(g);
    return b > m ? b : m;
}

// the step-by-step stage in parity blocks: a DNS group (the operators of a
// linear group need not be centro-symmetric) whose tiles fit
bool step_eo_supported(const GroupView& g) {
    return !g.lin && g.ny >= 3 && forcing_eo_smem_bytes(g) <= 227 * 1024 && helm_eo_smem_bytes(g) <= 227 * 1024;
}

void launch_forcing_eo(const GroupView& g, int s, cudaStream_t st) {
    gt::Tile t = gt::tile_of(g.E, g.ny, g.nmodes);
    dim3 grid((g.nmodes + t.QT - 1) / t.QT, (g.E + t.EBT - 1) / t.EBT);
    sto::k_forcing_eo<<<grid, sto::THREADS, forcing_eo_smem_bytes(g), st>>>(g, s);
}

void launch_helm_eo(const GroupView& g, int s, cudaStream_t st) {
    sto::k_helm_eo<<<mean_row_ctas(g) + 2 * g.npairs * helm_member_chunks(g), sto::THREADS, helm_eo_smem_bytes(g),
                     st>>>(g, s);
}

size_t yderiv_eo_smem_bytes(const GroupView& g) {
    const gt::Tile t = sto::yde_tile(g.E, g.ny, g.nmodes, g.yd_cap);
    const size_t b = sto::yde_bytes(g.ny, t.NC), m = mean_smem_bytes(g);
    return b > m ? b : m;
}

// the y-derivatives in parity blocks (D1 and D2 have the reflection symmetry on
// every group's interior grid, linear groups included)
bool yderiv_eo_supported(const GroupView& g) { return g.ny >= 3 && yderiv_eo_smem_bytes(g) <= 227 * 1024; }

void launch_yderiv_eo(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev) {
    const gt::Tile t = sto::yde_tile(g.E, g.ny, g.nmodes, g.yd_cap);
    dim3 grid((g.nmodes + t.QT - 1) / t.QT, (g.E + t.EBT - 1) / t.EBT);
    grid.y += mean_finish_extra_rows(g, grid.x, sprev);
    sto::k_yderiv_eo<<<grid, sto::THREADS, yderiv_eo_smem_bytes(g), st>>>(g, v, e, sprev);
}

void set_attributes_step_eo() {
    allow_max_dynamic_smem(sto::k_yderiv_eo);
    allow_max_dynamic_smem(sto::k_forcing_eo);
    allow_max_dynamic_smem(sto::k_helm_eo);
}

}  // namespace dnsk
