// Spectral-space kernels of one CN/RK3 sub-step (paper Sec. 3):
//   k_yderiv      Dv, D2v, D eta on the interior nodes (y-contraction with the
//                 shared Chebyshev operators, Sec. 3.1) and the H -> P relayout
//   k_forcing     F = -k^2 Nv - D(i kx Nu + i kz Nw), G = i kz Nu - i kx Nw
//                 (Eqs. Dv, eta) and the RK3 combination of Sec. 3.1
//   k_helm        x_s = M_h x_t + P_h F~ per wavenumber pair (Eqs. CN1, CN2),
//                 with M_1 x_t computed once and reused by sub-steps 2 and 3
//   k_mean_finish U00, W00 update (Eqs. CN3, CN4): the Poiseuille constant-flux
//                 gamma and the profiles, after the rows (mean.cuh) that run as
//                 extra CTAs of the implicit apply
//   k_stats_*     one-point statistics (Sec. 4)
//   k_pack/unpack host layout <-> H layout, Hermitian projection of n = 0
#include "dns_internal.hpp"
#include "mean.cuh"

namespace dnsk {

// ------------------------------------------------------------------ y-derivs

constexpr int QB = 8;   // modes per tile
constexpr int EB = 4;   // members per tile

// T is the arithmetic (and output) type: double for the FP64 path, float for
// the mixed path (the FP64 state is rounded to float on load).
template <typename T>
__global__ void __launch_bounds__(256) k_yderiv(const double2* __restrict__ v, const double2* __restrict__ et,
                                                const T* __restrict__ D1i, const T* __restrict__ D2i,
                                                typename C2<T>::type* __restrict__ P5, int Ny, int E, int nmodes,
                                                GroupView g, int sprev) {
    typedef typename C2<T>::type C;
    extern __shared__ __align__(16) unsigned char sm[];
    if (mean_finish_rows(g, sprev, (E + EB - 1) / EB, sm)) return;
    C* xv = (C*)sm;                 // [QB][Ny][EB]
    C* xe = xv + QB * Ny * EB;
    const int q0 = blockIdx.x * QB, e0 = blockIdx.y * EB;
    const int tile = QB * Ny * EB;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int ee = idx % EB;
        int y = (idx / EB) % Ny;
        int qq = idx / (EB * Ny);
        int q = q0 + qq, e = e0 + ee;
        C a = czero<C>(), b = a;
        if (q < nmodes && e < E) {
            size_t o = ((size_t)q * Ny + y) * E + e;
            double2 va = v[o], vb = et[o];
            a.x = (T)va.x; a.y = (T)va.y;
            b.x = (T)vb.x; b.y = (T)vb.y;
        }
        xv[idx] = a;
        xe[idx] = b;
    }
    __syncthreads();
    const size_t fs = (size_t)Ny * E * nmodes;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int qq = idx % QB;
        int ee = (idx / QB) % EB;
        int y = idx / (QB * EB);
        int q = q0 + qq, e = e0 + ee;
        T dvx = 0, dvy = 0, d2x = 0, d2y = 0, dex = 0, dey = 0;
        const T* r1 = D1i + (size_t)y * Ny;
        const T* r2 = D2i + (size_t)y * Ny;
        for (int k = 0; k < Ny; ++k) {
            T d1 = __ldg(r1 + k), d2 = __ldg(r2 + k);
            C a = xv[(qq * Ny + k) * EB + ee];
            C b = xe[(qq * Ny + k) * EB + ee];
            dvx += d1 * a.x; dvy += d1 * a.y;
            d2x += d2 * a.x; d2y += d2 * a.y;
            dex += d1 * b.x; dey += d1 * b.y;
        }
        if (q < nmodes && e < E) {
            size_t o = ((size_t)y * E + e) * nmodes + q;
            C a = xv[(qq * Ny + y) * EB + ee];
            C b = xe[(qq * Ny + y) * EB + ee];
            C c;
            P5[o] = a;
            c.x = dvx; c.y = dvy; P5[fs + o] = c;
            c.x = d2x; c.y = d2y; P5[2 * fs + o] = c;
            P5[3 * fs + o] = b;
            c.x = dex; c.y = dey; P5[4 * fs + o] = c;
        }
    }
}

template <typename T> __host__ __device__ const T* d1i_of(const GroupView& g);
template <> __host__ __device__ const double* d1i_of<double>(const GroupView& g) { return g.D1i; }
template <typename T> __host__ __device__ const T* d2i_of(const GroupView& g);
template <> __host__ __device__ const double* d2i_of<double>(const GroupView& g) { return g.D2i; }

template <typename T>
void launch_yderiv(const GroupView& g, const double2* v, const double2* e, void* P5, cudaStream_t st, int sprev) {
    dim3 grid((g.nmodes + QB - 1) / QB, (g.E + EB - 1) / EB);
    grid.y += mean_finish_extra_rows(g, grid.x, sprev);
    size_t smem = 2 * (size_t)QB * g.ny * EB * sizeof(typename C2<T>::type);
    k_yderiv<T><<<grid, 256, smem, st>>>(v, e, d1i_of<T>(g), d2i_of<T>(g), (typename C2<T>::type*)P5, g.ny, g.E,
                                         g.nmodes, g, sprev);
}
template void launch_yderiv<double>(const GroupView&, const double2*, const double2*, void*, cudaStream_t, int);

// ------------------------------------------------------------------- forcing

template <typename T>
__global__ void __launch_bounds__(256) k_forcing(GroupView g, int s) {
    typedef typename C2<T>::type C;
    extern __shared__ __align__(16) unsigned char sm[];
    C* phi = (C*)sm;   // [QB][Ny][EB], i kx Nu + i kz Nw in the arithmetic type T
    const T* D1 = d1i_of<T>(g);
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes, NKX = g.nkx;
    const int q0 = blockIdx.x * QB, e0 = blockIdx.y * EB;
    const int tile = QB * Ny * EB;
    const size_t fs = (size_t)Ny * E * nmodes;
    const C* N3 = (const C*)g.N3;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int qq = idx % QB;
        int ee = (idx / QB) % EB;
        int y = idx / (QB * EB);
        int q = q0 + qq, e = e0 + ee;
        C p = czero<C>();
        if (q < nmodes && e < E) {
            size_t o = ((size_t)y * E + e) * nmodes + q;
            C nu = N3[o], nw = N3[2 * fs + o];
            int mi = q / NKX, n = q - mi * NKX;
            T kx = (T)g.kxt[n], kz = (T)g.kzt[mi];
            // i kx Nu + i kz Nw
            T ax = kx * nu.x + kz * nw.x;
            T ay = kx * nu.y + kz * nw.y;
            p.x = -ay; p.y = ax;
        }
        phi[(qq * Ny + y) * EB + ee] = p;
    }
    __syncthreads();
    const int q_mean = mean_mode(g);
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int ee = idx % EB;
        int y = (idx / EB) % Ny;
        int qq = idx / (EB * Ny);
        int q = q0 + qq, e = e0 + ee;
        if (q >= nmodes || e >= E) continue;
        T tx = 0, ty = 0;
        const T* r1 = D1 + (size_t)y * Ny;
        for (int k = 0; k < Ny; ++k) {
            T d = __ldg(r1 + k);
            C p = phi[(qq * Ny + k) * EB + ee];
            tx += d * p.x; ty += d * p.y;
        }
        const double sx = (double)tx, sy = (double)ty;
        size_t o = ((size_t)y * E + e) * nmodes + q;
        C nu = N3[o], nv = N3[fs + o], nw = N3[2 * fs + o];
        int mi = q / NKX, n = q - mi * NKX;
        double kx = g.kxt[n], kz = g.kzt[mi], k2 = g.k2t[q];
        double2 F, G;
        F.x = -k2 * (double)nv.x - sx;
        F.y = -k2 * (double)nv.y - sy;
        // i kz Nu - i kx Nw
        double bx = kz * (double)nu.x - kx * (double)nw.x;
        double by = kz * (double)nu.y - kx * (double)nw.y;
        G = make_double2(-by, bx);
        if (q == q_mean) { F = make_double2(0.0, 0.0); G = F; }
        if (g.fn > 0 && n == g.fn) {   // stochastic forcing of the step
            const size_t o = ((size_t)mi * Ny + y) * E + e, half = (size_t)g.nkz * Ny * E;
            F.x += g.noise[o].x; F.y += g.noise[o].y;
            G.x += g.noise[half + o].x; G.y += g.noise[half + o].y;
        }
        size_t h = ((size_t)q * Ny + y) * E + e;
        double2 Ft, Gt;
        if (s == 0) {
            Ft = F; Gt = G;
            g.Av[h] = F; g.Ae[h] = G;
        } else if (s == 1) {
            double2 a = g.Av[h], b = g.Ae[h];
            Ft = make_double2(2.0 * F.x - a.x, 2.0 * F.y - a.y);
            Gt = make_double2(2.0 * G.x - b.x, 2.0 * G.y - b.y);
            g.Av[h] = make_double2((1.0 / 6.0) * a.x + (4.0 / 6.0) * F.x, (1.0 / 6.0) * a.y + (4.0 / 6.0) * F.y);
            g.Ae[h] = make_double2((1.0 / 6.0) * b.x + (4.0 / 6.0) * G.x, (1.0 / 6.0) * b.y + (4.0 / 6.0) * G.y);
        } else {
            double2 a = g.Av[h], b = g.Ae[h];
            Ft = make_double2(a.x + (1.0 / 6.0) * F.x, a.y + (1.0 / 6.0) * F.y);
            Gt = make_double2(b.x + (1.0 / 6.0) * G.x, b.y + (1.0 / 6.0) * G.y);
        }
        g.Fv[h] = Ft;
        g.Fe[h] = Gt;
    }
}

template <typename T>
void launch_forcing(const GroupView& g, int s, cudaStream_t st) {
    dim3 grid((g.nmodes + QB - 1) / QB, (g.E + EB - 1) / EB);
    size_t smem = (size_t)QB * g.ny * EB * sizeof(typename C2<T>::type);
    k_forcing<T><<<grid, 256, smem, st>>>(g, s);
}
template void launch_forcing<double>(const GroupView&, int, cudaStream_t);

// --------------------------------------------------------------------- mean

// Mean-flow update of every member (Eqs. CN3, CN4), one CTA per member.  It
// depends only on the plane means and the mean profiles, so it runs beside the
// forcing and implicit-apply kernels (own stream, joined before the next plane
// stage).
// The rows of every member run as leading CTAs of the implicit-apply launch
// (mean_rows, E x ceil(Ny / 8) CTAs, one warp per row); this kernel adds the
// constant-flux correction and writes the profiles, one CTA per member.
__global__ void __launch_bounds__(128) k_mean_finish(GroupView g, int s) {
    __shared__ double red[32];
    mean_finish(g, s, blockIdx.x, (unsigned char*)red);
    // the step's noise has been used by all three forcing assemblies: next step's
    if (s == 2 && g.fn > 0 && blockIdx.x == 0 && threadIdx.x == 0) *g.fstep += 1ULL;
}

void launch_mean_finish(const GroupView& g, int s, cudaStream_t st) {
    k_mean_finish<<<g.E, 128, 0, st>>>(g, s);
}

// --------------------------------------------------------------------- helm

// stage: the pair's two operators are copied to shared memory (they fit up to
// Ny = 120); above that every CTA reads them from global memory, where the
// 2 npairs x 2 operators stay L2-resident across the CTAs of the launch.
__global__ void __launch_bounds__(256) k_helm(GroupView g, int s, bool stage) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = g.ny, E = g.E, NKX = g.nkx;
    // leading CTAs: rows of the mean-flow update
    const int nrow = mean_row_ctas(g);
    if ((int)blockIdx.x < nrow) {
        mean_rows(g, s, blockIdx.x % E, (blockIdx.x / E) * (blockDim.x >> 5), sm);
        return;
    }
    const int b = blockIdx.x - nrow;
    const int p = b % g.npairs, f = (b / g.npairs) & 1, ch = b / (2 * g.npairs);
    const int n = p % NKX, am = p / NKX;
    if (!g.lin && n == 0 && am == 0) return;   // the mean mode (DNS groups)
    // members e0 .. e0 + ec - 1 (all of them unless the group is split into chunks)
    const int EC = helm_member_chunk(g), e0 = ch * EC, ec = min(EC, E - e0);
    const int hi = (s == 0) ? 0 : 1;
    const size_t nn = (size_t)Ny * Ny;
    const double* Mg = g.ops[hi] + ((size_t)p * 4 + (f == 0 ? 0 : 2)) * nn;
    const double* Pg = Mg + nn;
    const bool needM = (s != 2);
    const double* Ms = Mg;
    const double* Ps = Pg;
    if (stage) {
        double* ms = (double*)sm;
        double* ps = ms + nn;
        for (size_t i = threadIdx.x; i < nn; i += blockDim.x) {
            if (needM) ms[i] = Mg[i];
            ps[i] = Pg[i];
        }
        __syncthreads();
        Ms = ms;
        Ps = ps;
    }
    const int nq = am > 0 ? 2 : 1;
    const int q1 = (g.kz + am) * NKX + n, q2 = (g.kz - am) * NKX + n;
    const double2* X = f == 0 ? g.v_t : g.e_t;
    const double2* F = f == 0 ? g.Fv : g.Fe;
    double2* M1 = f == 0 ? g.mx1_v : g.mx1_e;
    double2* O = (s == 2) ? (f == 0 ? g.v_t : g.e_t) : (f == 0 ? g.v_s : g.e_s);
    const int ncol = 2 * E;                // real columns of a row in global memory
    const int per = Ny * 2 * ec;
    for (int idx = threadIdx.x; idx < nq * per; idx += blockDim.x) {
        int which = idx / per;
        int r = idx - which * per;
        int y = r / (2 * ec), c = 2 * e0 + r - y * (2 * ec);
        int q = which == 0 ? q1 : q2;
        const double* xc = (const double*)(X + (size_t)q * Ny * E);
        const double* fc = (const double*)(F + (size_t)q * Ny * E);
        double* m1 = (double*)(M1 + (size_t)q * Ny * E);
        double* oc = (double*)(O + (size_t)q * Ny * E);
        double accP = 0.0;
        const double* pr = Ps + (size_t)y * Ny;
        for (int k = 0; k < Ny; ++k) accP += pr[k] * fc[k * ncol + c];
        double out;
        if (needM) {
            double accM = 0.0;
            const double* mr = Ms + (size_t)y * Ny;
            for (int k = 0; k < Ny; ++k) accM += mr[k] * xc[k * ncol + c];
            if (s == 1) m1[y * ncol + c] = accM;
            out = accM + accP;
        } else {
            out = m1[y * ncol + c] + accP;
        }
        oc[y * ncol + c] = out;
    }
}

void launch_helm(const GroupView& g, int s, cudaStream_t st) {
    size_t smem = 2 * (size_t)g.ny * g.ny * sizeof(double);
    const bool stage = smem <= 227 * 1024;
    if (!stage) smem = 0;
    if (smem < mean_smem_bytes(g)) smem = mean_smem_bytes(g);
    k_helm<<<mean_row_ctas(g) + 2 * g.npairs * helm_member_chunks(g), 256, smem, st>>>(g, s, stage);
}


// --------------------------------------------------------------------- mean

// -------------------------------------------------------------------- stats

// Per-plane Parseval sums of one (interior plane y, member e) into part[e][y][6]:
// uu, vv, ww, uv (perturbation, Sec. 4), max |div u|, non-finite flag.
__global__ void __launch_bounds__(256) k_stats_plane(GroupView g, double* __restrict__ part) {
    __shared__ double red[32];
    const int y = blockIdx.x, e = blockIdx.y;
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes, NKX = g.nkx;
    const size_t fs = (size_t)Ny * E * nmodes;
    const double2* P = g.P5d + ((size_t)y * E + e) * nmodes;
    double uu = 0, vv = 0, ww = 0, uv = 0, dmax = 0, nf = 0;
    const int q_mean = mean_mode(g);
    for (int q = threadIdx.x; q < nmodes; q += blockDim.x) {
        double2 v = P[q], dv = P[fs + q], et = P[3 * fs + q];
        if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(et.x) || !isfinite(et.y)) nf = 1.0;
        if (q == q_mean) continue;
        int mi = q / NKX, n = q - mi * NKX;
        double kx = g.kxt[n], kz = g.kzt[mi], ki = g.k2inv[q];
        // u = i (kx Dv - kz eta) / k^2, w = i (kz Dv + kx eta) / k^2
        double ax = (kx * dv.x - kz * et.x) * ki, ay = (kx * dv.y - kz * et.y) * ki;
        double bx = (kz * dv.x + kx * et.x) * ki, by = (kz * dv.y + kx * et.y) * ki;
        double2 u = make_double2(-ay, ax), w = make_double2(-by, bx);
        double c = (n == 0 || g.lin) ? 1.0 : 2.0;   // real fields carry -kx too
        uu += c * (u.x * u.x + u.y * u.y);
        vv += c * (v.x * v.x + v.y * v.y);
        ww += c * (w.x * w.x + w.y * w.y);
        uv += c * (u.x * v.x + u.y * v.y);
        // i kx u + Dv + i kz w
        double rx = -kx * u.y + dv.x - kz * w.y;
        double ry = kx * u.x + dv.y + kz * w.x;
        dmax = fmax(dmax, sqrt(rx * rx + ry * ry));
    }
    uu = block_sum(uu, red); vv = block_sum(vv, red); ww = block_sum(ww, red);
    uv = block_sum(uv, red); dmax = block_max(dmax, red); nf = block_max(nf, red);
    if (threadIdx.x == 0) {
        double* o = part + ((size_t)e * Ny + y) * 6;
        o[0] = uu; o[1] = vv; o[2] = ww; o[3] = uv; o[4] = dmax; o[5] = nf;
    }
}

// CFL rate of one interior plane (y, e), without the factor dt: the maximum over
// the plane's Mx x Mz collocation points of |u|/dx + |v|/dy + |w|/dz, mean flow
// included, dy the smaller gap from the node to a neighbour.  u, v, w come from
// the FP64 spectra of the statistics pass (v, Dv, eta of P5d; u, w by the
// explicit solutions, Sec. 3.2) and are synthesised on the grid in single
// precision by direct sums, along z for every kept kx, then along x (the kx = 0
// column entering by its real part, every other column twice).
__global__ void __launch_bounds__(256) k_stats_cfl(GroupView g) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float red[32];
    const int y = blockIdx.x, e = blockIdx.y;
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes, NKX = g.nkx, NKZ = g.nkz, Kz = g.kz;
    const int Mx = g.mx, Mz = g.mz, My = g.my, jn = y + 1;
    float2* c = (float2*)sm;                   // [NKZ][NKX] coefficients of one field
    float2* s = c + nmodes;                    // [NKX][Mz] after the z sums
    float2* tz = s + (size_t)NKX * Mz;         // exp(2 pi i k / Mz)
    float2* tx = tz + Mz;                      // exp(2 pi i k / Mx)
    float* acc = (float*)(tx + Mx);            // [Mz][Mx] rate of every point
    for (int k = threadIdx.x; k < Mz; k += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * k / Mz, &sn, &cs);
        tz[k] = make_float2((float)cs, (float)sn);
    }
    for (int k = threadIdx.x; k < Mx; k += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * k / Mx, &sn, &cs);
        tx[k] = make_float2((float)cs, (float)sn);
    }
    const double yj = -cospi((double)jn / (My - 1));
    const double dy = fmin(yj + cospi((double)(jn - 1) / (My - 1)), -cospi((double)(jn + 1) / (My - 1)) - yj);
    const size_t fs = (size_t)Ny * E * nmodes;
    const double2* P = g.P5d + ((size_t)y * E + e) * nmodes;
    const int q_mean = mean_mode(g);
    for (int f = 0; f < 3; ++f) {   // u, v, w
        const float inv = (float)(f == 0 ? Mx / g.lx : f == 1 ? 1.0 / dy : Mz / g.lz);
        __syncthreads();   // the previous field's sums are done with c and s
        for (int q = threadIdx.x; q < nmodes; q += blockDim.x) {
            double2 val;
            if (q == q_mean) {
                val = make_double2(f == 0 ? g.U_t[(size_t)e * My + jn] : f == 2 ? g.W_t[(size_t)e * My + jn] : 0.0,
                                   0.0);
            } else if (f == 1) {
                val = P[q];
            } else {
                // u = i (kx Dv - kz eta) / k^2, w = i (kz Dv + kx eta) / k^2
                const int mi = q / NKX, n = q - mi * NKX;
                const double kx = g.kxt[n], kz = g.kzt[mi], ki = g.k2inv[q];
                const double a = f == 0 ? kx : kz, b = f == 0 ? -kz : kx;
                const double2 dv = P[fs + q], et = P[3 * fs + q];
                val = make_double2(-(a * dv.y + b * et.y) * ki, (a * dv.x + b * et.x) * ki);
            }
            c[q] = make_float2((float)val.x, (float)val.y);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < NKX * Mz; idx += blockDim.x) {
            const int n = idx / Mz, k = idx - n * Mz;
            float sr = 0.f, si = 0.f;
            for (int mi = 0; mi < NKZ; ++mi) {
                int r = ((mi - Kz) * k) % Mz;
                if (r < 0) r += Mz;
                const float2 a = c[mi * NKX + n], t = tz[r];
                sr += a.x * t.x - a.y * t.y;
                si += a.x * t.y + a.y * t.x;
            }
            s[idx] = make_float2(sr, si);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < Mz * Mx; idx += blockDim.x) {
            const int k = idx / Mx, i = idx - k * Mx;
            float sum = 0.f;
            for (int n = 1; n < NKX; ++n) {
                const float2 a = s[n * Mz + k], t = tx[(n * i) % Mx];
                sum += a.x * t.x - a.y * t.y;
            }
            const float r = fabsf(s[k].x + 2.f * sum) * inv;
            acc[idx] = f == 0 ? r : acc[idx] + r;   // the same thread owns idx for every field
        }
    }
    float mx = 0.f;
    for (int idx = threadIdx.x; idx < Mz * Mx; idx += blockDim.x) mx = fmaxf(mx, acc[idx]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) g.cfl_y[(size_t)e * Ny + y] = (double)v;
    }
}

size_t stats_cfl_smem_bytes(const GroupView& g) {
    return sizeof(float2) * ((size_t)g.nmodes + (size_t)g.nkx * g.mz + g.mz + g.mx) +
           sizeof(float) * (size_t)g.mz * g.mx;
}

// Per-member reduction over y (Clenshaw-Curtis weights) of the plane sums in
// part, packed into out[e][ostride]: e_total, e_pert, tau_bottom, tau_top,
// bulk_flux, gamma, max_div, nonfinite and, with full, the CFL number (then
// ostride >= 9), the profiles going to g.prof.  Without full only the first
// eight values are written and neither the profiles nor the CFL rates are read.
__global__ void k_stats_final(GroupView g, const double* __restrict__ part, double* __restrict__ out, int ostride,
                              int full) {
    __shared__ double red[32];
    const int e = blockIdx.x, Ny = g.ny, My = g.my;
    const double* U = g.U_t + (size_t)e * My;
    const double* W = g.W_t + (size_t)e * My;
    double* prof = full ? g.prof + (size_t)e * 6 * My : nullptr;
    double ep = 0, em = 0, fl = 0, dm = 0, nf = 0, cf = 0;
    for (int j = threadIdx.x; j < My; j += blockDim.x) {
        double uu = 0, vv = 0, ww = 0, uv = 0;
        if (j > 0 && j < My - 1) {
            const double* s = part + ((size_t)e * Ny + (j - 1)) * 6;
            uu = s[0]; vv = s[1]; ww = s[2]; uv = s[3];
            dm = fmax(dm, s[4]);
            nf = fmax(nf, s[5]);
            if (full && !g.lin) cf = fmax(cf, g.cfl_y[(size_t)e * Ny + (j - 1)]);
        }
        if (!isfinite(U[j]) || !isfinite(W[j])) nf = 1.0;
        if (prof) {
            prof[0 * My + j] = U[j];
            prof[1 * My + j] = W[j];
            prof[2 * My + j] = uu;
            prof[3 * My + j] = vv;
            prof[4 * My + j] = ww;
            prof[5 * My + j] = uv;
        }
        double w = g.ccw[j];
        ep += w * (uu + vv + ww);
        em += w * (U[j] * U[j] + W[j] * W[j]);
        fl += w * U[j];
    }
    ep = block_sum(ep, red); em = block_sum(em, red); fl = block_sum(fl, red);
    dm = block_max(dm, red); nf = block_max(nf, red); cf = block_max(cf, red);
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0;
        for (int j = 0; j < My; ++j) {
            t0 += g.D1[j] * U[j];
            t1 += g.D1[(size_t)(My - 1) * My + j] * U[j];
        }
        double* o = out + (size_t)e * ostride;
        o[0] = 0.25 * (ep + em);
        o[1] = 0.25 * ep;
        o[2] = t0;
        o[3] = t1;
        o[4] = fl;
        o[5] = g.gamma[e];
        o[6] = dm;
        o[7] = nf;
        if (full) o[8] = cf * g.dt;
    }
}

// Shared-mean (S3T-type) ensemble, Sec. 4.1: the kx = 0 column of the three
// nonlinear terms (P layout, n = 0 of every m and interior plane) and the plane
// means <uv>, <wv> are replaced by their average over the members, summed in
// member order.  One thread per averaged quantity.
template <typename C>
__global__ void k_shared_mean(GroupView g) {
    const int E = g.E, Ny = g.ny, NM = g.nmodes, NKX = g.nkx, My = g.my;
    const int nN = 3 * Ny * g.nkz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nN) {
        const int mi = t % g.nkz, r = t / g.nkz, y = r % Ny, f = r / Ny;
        C* p = (C*)g.N3 + (size_t)f * Ny * E * NM + (size_t)y * E * NM + (size_t)mi * NKX;
        C acc = p[0];
        for (int e = 1; e < E; ++e) {
            acc.x += p[(size_t)e * NM].x;
            acc.y += p[(size_t)e * NM].y;
        }
        acc.x /= E;
        acc.y /= E;
        for (int e = 0; e < E; ++e) p[(size_t)e * NM] = acc;
    } else if (t < nN + 2 * Ny) {
        const int j = t - nN, y = 1 + j % Ny;
        double* m = (j < Ny) ? g.uv : g.wv;
        double acc = m[y];
        for (int e = 1; e < E; ++e) acc += m[(size_t)e * My + y];
        acc /= E;
        for (int e = 0; e < E; ++e) m[(size_t)e * My + y] = acc;
    }
}

void launch_shared_mean(const GroupView& g, bool fp64, cudaStream_t st) {
    const int n = 3 * g.ny * g.nkz + 2 * g.ny;
    const int th = 256, bl = (n + th - 1) / th;
    if (fp64) k_shared_mean<double2><<<bl, th, 0, st>>>(g);
    else k_shared_mean<float2><<<bl, th, 0, st>>>(g);
}

void launch_stats(const GroupView& g, cudaStream_t st) {
    launch_yderiv<double>(g, g.v_t, g.e_t, g.P5d, st);
    k_stats_plane<<<dim3(g.ny, g.E), 256, 0, st>>>(g, g.st_y);
    if (!g.lin) k_stats_cfl<<<dim3(g.ny, g.E), 256, stats_cfl_smem_bytes(g), st>>>(g);
    k_stats_final<<<g.E, 128, 0, st>>>(g, g.st_y, g.st_out, 9, 1);
}

void launch_stats_packed(const GroupView& g, double* part, double* out, cudaStream_t st) {
    launch_yderiv<double>(g, g.v_t, g.e_t, g.P5d, st);
    k_stats_plane<<<dim3(g.ny, g.E), 256, 0, st>>>(g, part);
    k_stats_final<<<g.E, 128, 0, st>>>(g, part, out, 8, 0);
}

// --------------------------------------------------------------- pack/unpack

// Host layout -> H layout.  sv, se: v and eta, each [count][Ny][NKZ][NKX]
// complex; sU, sW: [count][My] (nullptr: the profiles were copied separately).
// The sources are device memory, the host-layout staging buffer, or page-locked
// host memory mapped into the device's address space (read over the CPU-GPU
// link; no intermediate copy).
constexpr int TRANSFER_BOUND = 64;   // threads per CTA of the transfer kernels (at most)
__global__ void __launch_bounds__(TRANSFER_BOUND) k_pack(GroupView g, int member0, int count,
                                                         const double2* __restrict__ sv,
                                                         const double2* __restrict__ se, const double* __restrict__ sU,
                                                         const double* __restrict__ sW) {
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes, NKX = g.nkx, NKZ = g.nkz;
    const size_t per = (size_t)count * Ny * nmodes;
    const int q_mean = mean_mode(g);
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
    for (size_t idx = t0; idx < per; idx += nt) {
        int q = (int)(idx % nmodes);
        int y = (int)((idx / nmodes) % Ny);
        int el = (int)(idx / ((size_t)nmodes * Ny));
        int mi = q / NKX, n = q - mi * NKX;
        double2 a = sv[idx], b = se[idx];
        if (n == 0 && !g.lin) {
            // Hermitian part of the n = 0 column: (x(m) + conj x(-m)) / 2
            int qp = (NKZ - 1 - mi) * NKX;
            size_t ip = ((size_t)el * Ny + y) * nmodes + qp;
            double2 ap = sv[ip], bp = se[ip];
            a = make_double2(0.5 * (a.x + ap.x), 0.5 * (a.y - ap.y));
            b = make_double2(0.5 * (b.x + bp.x), 0.5 * (b.y - bp.y));
        }
        if (q == q_mean) { a = make_double2(0.0, 0.0); b = a; }
        if (!DNS_CK(g.status, member0 + el < E, CK_PACK, idx)) continue;
        size_t h = ((size_t)q * Ny + y) * E + member0 + el;
        g.v_t[h] = a;
        g.e_t[h] = b;
    }
    if (sU) {
        const size_t nu = (size_t)count * g.my, o = (size_t)member0 * g.my;
        for (size_t i = t0; i < nu; i += nt) {
            if (!DNS_CK(g.status, o + i < (size_t)E * g.my, CK_PACK, i)) continue;
            g.U_t[o + i] = sU[i];
            g.W_t[o + i] = sW[i];
        }
    }
}

// H layout -> host layout, into device memory, the staging buffer or mapped
// page-locked host memory (written over the CPU-GPU link).  Any destination may
// be nullptr (not wanted).
__global__ void __launch_bounds__(TRANSFER_BOUND) k_unpack(GroupView g, int member0, int count,
                                                           double2* __restrict__ dv, double2* __restrict__ de,
                         double* __restrict__ dU, double* __restrict__ dW) {
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes;
    const size_t per = (size_t)count * Ny * nmodes;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
    for (size_t idx = t0; idx < per; idx += nt) {
        int q = (int)(idx % nmodes);
        int y = (int)((idx / nmodes) % Ny);
        int el = (int)(idx / ((size_t)nmodes * Ny));
        if (!DNS_CK(g.status, member0 + el < E, CK_UNPACK, idx)) continue;
        size_t h = ((size_t)q * Ny + y) * E + member0 + el;
        if (dv) dv[idx] = g.v_t[h];
        if (de) de[idx] = g.e_t[h];
    }
    const size_t nu = (size_t)count * g.my, o = (size_t)member0 * g.my;
    for (size_t i = t0; i < nu; i += nt) {
        if (!DNS_CK(g.status, o + i < (size_t)E * g.my, CK_UNPACK, i)) continue;
        if (dU) dU[i] = g.U_t[o + i];
        if (dW) dW[i] = g.W_t[o + i];
    }
}

// Small CTAs, three per SM: about 0.9 MB of reads in flight keeps the CPU-GPU
// link busy (a larger grid moves the data no faster), and CTAs of 64 threads x
// 32 registers still fit beside the step kernels of the member blocks that
// compute meanwhile (a line-owned plane CTA leaves 7936 of the SM's 65536
// registers: room for three; three implicit-apply CTAs leave 4096: two).
constexpr int TRANSFER_THREADS = TRANSFER_BOUND;
static int transfer_ctas() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = 3 * (sms > 0 ? sms : 1);
    }
    return n;
}

void launch_pack(const GroupView& g, int member0, int count, const double2* sv, const double2* se, const double* sU,
                 const double* sW, cudaStream_t st) {
    k_pack<<<transfer_ctas(), TRANSFER_THREADS, 0, st>>>(g, member0, count, sv, se, sU, sW);
}
void launch_unpack(const GroupView& g, int member0, int count, double2* dv, double2* de, double* dU, double* dW,
                   cudaStream_t st) {
    k_unpack<<<transfer_ctas(), TRANSFER_THREADS, 0, st>>>(g, member0, count, dv, de, dU, dW);
}

cudaError_t load_stats_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void*)k_stats_plane);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void*)k_stats_final);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void*)k_yderiv<double>);
    return e;
}

void set_attributes_spectral() {
    allow_max_dynamic_smem(k_stats_cfl);
    allow_max_dynamic_smem(k_yderiv<double>);
    allow_max_dynamic_smem(k_forcing<double>);
    allow_max_dynamic_smem(k_helm);
}

}  // namespace dnsk
