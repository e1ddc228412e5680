// Mean-flow update of one member, shared by the implicit-apply kernels.
#pragma once
#include "dns_internal.hpp"

namespace dnsk {

// Mean-flow update of every member (Eqs. CN3, CN4).  The forcing d/dy <uv> is
// folded into the solve (PD = PU D1), so the RK3 combination acts on the plane
// means themselves:
//   U_int = MU U_int + PD <uv>~ + bU [U(-1), U(+1)] (+ gamma Ug, Poiseuille),
// each row one warp with a lane-strided sum and a fixed shuffle tree.  The rows
// are spread over many SMs (the FP64 pipe of one SM is slow):
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// mean_rows, E x ceil(Ny / 8) extra CTAs of the implicit-apply launch, one warp
// per interior row i, writes
// the pre-gamma profiles Un, Wn (interior rows) to the scratch rows dU, dW.
// mean_finish, one CTA per member, adds gamma Ug (Poiseuille), writes the
// profiles and advances the RK accumulators of <uv>, <wv> (after every row CTA
// has read them).
__device__ __forceinline__ void mean_rows(const GroupView& g, int s, int e, int row0, unsigned char* sm) {
    const int Ny = g.ny, My = g.my;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* Ut = (double*)sm;       // [My] each
    double* Wt = Ut + My;
    double* cu = Wt + My;
    double* cw = cu + My;
    const int hi = (s == 0) ? 0 : 1;
    const double* MU = g.mops[hi];
    const double* PU = MU + (size_t)Ny * Ny;
    const double* bU = PU + (size_t)Ny * Ny;
    const double* Ug = bU + 2 * (size_t)Ny;
    const double* PD = Ug + Ny;
    for (int j = threadIdx.x; j < My; j += blockDim.x) {
        const size_t o = (size_t)e * My + j;
        const double a = g.uv[o], b = g.wv[o];
        Ut[j] = g.U_t[o];
        Wt[j] = g.W_t[o];
        double ca, cb;
        if (s == 0) {
            ca = a; cb = b;
        } else if (s == 1) {
            const double pa = g.AU[o], pb = g.AW[o];
            ca = 2.0 * a - pa; cb = 2.0 * b - pb;
        } else {
            ca = g.AU[o] + (1.0 / 6.0) * a;
            cb = g.AW[o] + (1.0 / 6.0) * b;
        }
        cu[j] = ca;
        cw[j] = cb;
    }
    __syncthreads();
    const int i = row0 + warp;
    if (warp < nw && i < Ny) {
        const double* mr = MU + (size_t)i * Ny;
        const double* pr = PD + (size_t)i * My;
        double a = 0.0, c = 0.0;
        for (int j = lane; j < Ny; j += 32) { a += mr[j] * Ut[j + 1]; c += mr[j] * Wt[j + 1]; }
        for (int j = lane; j < My; j += 32) { a += pr[j] * cu[j]; c += pr[j] * cw[j]; }
        a = warp_sum(a);
        c = warp_sum(c);
        if (lane == 0) {
            g.dU[(size_t)e * My + i + 1] = a + (bU[2 * i] * Ut[0] + bU[2 * i + 1] * Ut[My - 1]);
            g.dW[(size_t)e * My + i + 1] = c + (bU[2 * i] * Wt[0] + bU[2 * i + 1] * Wt[My - 1]);
        }
    }
}

__device__ __forceinline__ void mean_finish(const GroupView& g, int s, int e, unsigned char* sm) {
    const int Ny = g.ny, My = g.my;
    double* red = (double*)sm;     // [32]
    const int hi = (s == 0) ? 0 : 1;
    const double* Ug = g.mops[hi] + 2 * (size_t)Ny * Ny + 2 * (size_t)Ny;
    const double* Un = g.dU + (size_t)e * My;
    const double* Wn = g.dW + (size_t)e * My;
    const double* Ut = g.U_t + (size_t)e * My;
    const double* Wt = g.W_t + (size_t)e * My;
    // walls keep their values
    double gam = 0.0;
    if (g.flow == 1) {
        double fl = 0.0, fg = 0.0;
        for (int j = threadIdx.x; j < My; j += blockDim.x)
            fl += g.ccw[j] * ((j > 0 && j < My - 1) ? Un[j] : Ut[j]);
        for (int i = threadIdx.x; i < Ny; i += blockDim.x) fg += g.ccw[i + 1] * Ug[i];
        fl = block_sum(fl, red);
        fg = block_sum(fg, red);
        gam = (g.bulk_flux - fl) / fg;
    }
    double* Uo = (s == 2) ? (g.U_t + (size_t)e * My) : (g.U_s + (size_t)e * My);
    double* Wo = (s == 2) ? (g.W_t + (size_t)e * My) : (g.W_s + (size_t)e * My);
    // in sub-step 3 the output overwrites U_t: read every wall value first
    const double u0 = Ut[0], u1 = Ut[My - 1], w0 = Wt[0], w1 = Wt[My - 1];
    __syncthreads();
    for (int j = threadIdx.x; j < My; j += blockDim.x) {
        const bool wall = (j == 0 || j == My - 1);
        Uo[j] = wall ? (j == 0 ? u0 : u1) : Un[j] + gam * Ug[j - 1];
        Wo[j] = wall ? (j == 0 ? w0 : w1) : Wn[j];
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
}

// The finish of sub-steps 1 and 2 rides on the next sub-step's y-derivative
// launch (it is independent of it and done before the plane stage reads the
// profiles): grid rows gy0 and beyond of that 2-D launch hold one CTA per
// member, row-major over the grid's x extent.  True for those CTAs (which then
// return without touching the y-derivative work).
__device__ __forceinline__ bool mean_finish_rows(const GroupView& g, int sprev, int gy0, unsigned char* sm) {
    if (sprev < 0 || (int)blockIdx.y < gy0) return false;
    const int e = ((int)blockIdx.y - gy0) * (int)gridDim.x + (int)blockIdx.x;
    if (e < g.E) mean_finish(g, sprev, e, sm);
    return true;
}

inline int mean_finish_extra_rows(const GroupView& g, int gx, int sprev) {
    return sprev < 0 ? 0 : (g.E + gx - 1) / gx;
}

}  // namespace dnsk
