// Linearised disturbance ensembles about a frozen streamwise-mean base flow
// (paper, "Diagnostic utilities that benefit from vectorization" and "Growth
// functional and linearized adjoint equations of streamwise-mean flow
// dynamics").  A linear group holds one streamwise wavenumber kx != 0 and every
// kept kz; its members are disturbance vectors.  The y-derivative, forcing and
// implicit-apply stages are the DNS's own kernels (one kx column, no mean
// mode); this file holds what differs:
//
//   * the physical-space stage: for one interior plane of one member, the nine
//     fields u, v, w, d_y(u, v, w), d_z(u, v, w) are inverse-transformed along
//     z only (the x dependence is the single harmonic exp(i kx x), so d_x is a
//     factor i kx), multiplied with the base flow B = (U, V, W)(y, z) and its
//     derivatives, and the three products are transformed back and truncated:
//       forward  N_i = i kx U u_i + V d_y u_i + W d_z u_i + v d_y B_i + w d_z B_i
//                     ((B . grad) u' + (u' . grad) B),
//       adjoint  N_i = -(i kx U l_i + V d_y l_i + W d_z l_i) + sum_k l_k d_i B_k
//                     (-(B . grad) l + (grad B)^T l, no x-derivative of B),
//     the equations reading d/dt = -N - grad p + (1/Re) lap in both directions
//     (the adjoint runs in reversed time); the direction is read from device
//     memory at every launch, so a captured step graph serves both;
//   * modified Gram-Schmidt of the member set in the energy inner product
//     <a, b> = (1/4) sum_q sum_j w_j (conj(v_a) v_b + (conj(Dv_a) Dv_b +
//     conj(eta_a) eta_b) / k^2) over the interior nodes (w_j Clenshaw-Curtis
//     weights, Dv = D1 v with v = 0 at the walls): one launch per vector k
//     projects x_k out of every later vector (one CTA each) and normalises
//     x_{k-1}, whose projections the previous launch completed.
#include "dns_internal.hpp"

namespace dnsk {

constexpr int GS_THREADS = 256;

// threads of the plane stage for transforms of length MZ: one per butterfly of
// the widest stage over the nine lines (at most 320)
__host__ __device__ constexpr int lin_threads(int MZ) {
    int nb = 0;
    for (int s = 0; s < ct_stages(MZ); ++s) nb = MZ / ct_radix(MZ, s) > nb ? MZ / ct_radix(MZ, s) : nb;
    int t = 9 * nb;
    t = t > 320 ? 320 : t;
    return (t + 31) / 32 * 32;
}

template <typename T> struct LinTab;
template <> struct LinTab<double> {
    static __device__ __forceinline__ const double2* tw(const GroupView& g) { return g.twz; }
    static __device__ __forceinline__ const double* base(const GroupView& g) { return g.base; }
    static __device__ __forceinline__ const double* k2i(const GroupView& g) { return g.k2inv; }
    static __device__ __forceinline__ const double* kz(const GroupView& g) { return g.kzt; }
};
template <> struct LinTab<float> {
    static __device__ __forceinline__ const float2* tw(const GroupView& g) { return g.twzf; }
    static __device__ __forceinline__ const float* base(const GroupView& g) { return g.basef; }
    static __device__ __forceinline__ const float* k2i(const GroupView& g) { return g.k2invf; }
    static __device__ __forceinline__ const float* kz(const GroupView& g) { return g.kztf; }
};

template <typename T>
size_t lin_plane_smem_bytes(int mz) {
    return 2 * 9 * (size_t)mz * sizeof(typename C2<T>::type);
}

// i * (a x + b y) for complex x, y and real a, b
template <typename C, typename T>
__device__ __forceinline__ C i_lin2(T a, C x, T b, C y) {
    C r;
    r.x = -(a * x.y + b * y.y);
    r.y = a * x.x + b * y.x;
    return r;
}

template <typename C, typename T>
__device__ __forceinline__ C axpy3(T a, C x, T b, C y, T c, C z) {
    C r;
    r.x = a * x.x + b * y.x + c * z.x;
    r.y = a * x.y + b * y.y + c * z.y;
    return r;
}

template <typename T, int MZ>
__global__ void __launch_bounds__(lin_threads(MZ)) k_lin_plane(GroupView g) {
    typedef typename C2<T>::type C;
    extern __shared__ __align__(16) unsigned char sm[];
    const int y = blockIdx.x, e = blockIdx.y;
    constexpr int Mz = MZ;
    const int Ny = g.ny, E = g.E, NM = g.nmodes, Kz = g.kz;
    C* b0 = (C*)sm;
    C* b1 = b0 + 9 * Mz;
    const bool adjoint = *g.dir != 0;
    const size_t fs = (size_t)Ny * E * NM;
    const C* P = (const C*)g.P5 + ((size_t)y * E + e) * NM;
    const T kx = (T)g.kxt[0];
    const T* kzt = LinTab<T>::kz(g);
    const T* k2i = LinTab<T>::k2i(g);
    for (int i = threadIdx.x; i < 9 * Mz; i += blockDim.x) b0[i] = czero<C>();
    __syncthreads();
    // zero-padded spectral lines: u, v, w | d_y u, d_y v, d_y w | d_z u, d_z v, d_z w
    for (int q = threadIdx.x; q < NM; q += blockDim.x) {
        const int m = q - Kz, pos = m >= 0 ? m : m + Mz;
        const C v = P[q], dv = P[fs + q], d2v = P[2 * fs + q], et = P[3 * fs + q], de = P[4 * fs + q];
        const T kz = kzt[q], ki = k2i[q];
        // u = i (kx Dv - kz eta) / k^2, w = i (kz Dv + kx eta) / k^2
        const C u = cscale(i_lin2(kx, dv, -kz, et), ki);
        const C w = cscale(i_lin2(kz, dv, kx, et), ki);
        const C uy = cscale(i_lin2(kx, d2v, -kz, de), ki);
        const C wy = cscale(i_lin2(kz, d2v, kx, de), ki);
        b0[0 * Mz + pos] = u;
        b0[1 * Mz + pos] = v;
        b0[2 * Mz + pos] = w;
        b0[3 * Mz + pos] = uy;
        b0[4 * Mz + pos] = dv;
        b0[5 * Mz + pos] = wy;
        b0[6 * Mz + pos] = cscale(cmuli(u), kz);
        b0[7 * Mz + pos] = cscale(cmuli(v), kz);
        b0[8 * Mz + pos] = cscale(cmuli(w), kz);
    }
    __syncthreads();
    C* ph = fft_lines_ct<C, +1, MZ, 9>(b0, b1, LinTab<T>::tw(g));
    // products at every z (one thread reads the nine values at z and writes the
    // three results there)
    const T* B = LinTab<T>::base(g) + (size_t)y * Mz;
    const size_t bs = (size_t)Ny * Mz;
    for (int z = threadIdx.x; z < Mz; z += blockDim.x) {
        C a[9];
#pragma unroll
        for (int f = 0; f < 9; ++f) a[f] = ph[f * Mz + z];
        const T U = B[z], V = B[bs + z], W = B[2 * bs + z];
        const T By[3] = {B[3 * bs + z], B[4 * bs + z], B[5 * bs + z]};
        const T Bz[3] = {B[6 * bs + z], B[7 * bs + z], B[8 * bs + z]};
        C N[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // (B . grad) a_i = i kx U a_i + V d_y a_i + W d_z a_i
            C adv = cscale(cmuli(a[i]), kx * U);
            adv.x += V * a[3 + i].x + W * a[6 + i].x;
            adv.y += V * a[3 + i].y + W * a[6 + i].y;
            if (!adjoint) {
                N[i].x = adv.x + a[1].x * By[i] + a[2].x * Bz[i];
                N[i].y = adv.y + a[1].y * By[i] + a[2].y * Bz[i];
            } else if (i == 0) {
                N[i].x = -adv.x;
                N[i].y = -adv.y;
            } else {
                const C t = (i == 1) ? axpy3(By[0], a[0], By[1], a[1], By[2], a[2])
                                     : axpy3(Bz[0], a[0], Bz[1], a[1], Bz[2], a[2]);
                N[i].x = t.x - adv.x;
                N[i].y = t.y - adv.y;
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) ph[i * Mz + z] = N[i];
    }
    __syncthreads();
    C* out = fft_lines_ct<C, -1, MZ, 3>(ph, ph == b0 ? b1 : b0, LinTab<T>::tw(g));
    // keep |m| <= Kz; the forward transform carries 1/Mz
    const T sc = (T)(1.0 / (double)Mz);
    C* N3 = (C*)g.N3 + ((size_t)y * E + e) * NM;
    for (int i = threadIdx.x; i < 3 * NM; i += blockDim.x) {
        const int f = i / NM, q = i - f * NM, m = q - Kz, pos = m >= 0 ? m : m + Mz;
        N3[(size_t)f * fs + q] = cscale(out[f * Mz + pos], sc);
    }
}

template <typename T, int MZ>
void launch_lin_plane_t(const GroupView& g, cudaStream_t st) {
    k_lin_plane<T, MZ><<<dim3(g.ny, g.E), lin_threads(MZ), lin_plane_smem_bytes<T>(MZ), st>>>(g);
}

template <typename T>
void launch_lin_plane_p(const GroupView& g, cudaStream_t st) {
    switch (g.mz) {   // the spanwise sizes a group accepts
        case 16: launch_lin_plane_t<T, 16>(g, st); break;
        case 32: launch_lin_plane_t<T, 32>(g, st); break;
        case 48: launch_lin_plane_t<T, 48>(g, st); break;
        case 64: launch_lin_plane_t<T, 64>(g, st); break;
        default: launch_lin_plane_t<T, 128>(g, st); break;
    }
}

void launch_lin_plane(const GroupView& g, bool fp64, cudaStream_t st) {
    if (fp64) launch_lin_plane_p<double>(g, st);
    else launch_lin_plane_p<float>(g, st);
}

// ------------------------------------------------------------ Gram-Schmidt

// Dv = D1_int v for every member and kz (H layout, into the v_s scratch field)
__global__ void __launch_bounds__(GS_THREADS) k_lin_dv(GroupView g) {
    extern __shared__ __align__(16) unsigned char sm[];
    double* D = (double*)sm;
    const int Ny = g.ny, E = g.E, q = blockIdx.x;
    for (int i = threadIdx.x; i < Ny * Ny; i += blockDim.x) D[i] = g.D1i[i];
    __syncthreads();
    const double2* v = g.v_t + (size_t)q * Ny * E;
    double2* o = g.v_s + (size_t)q * Ny * E;
    for (int i = threadIdx.x; i < Ny * E; i += blockDim.x) {
        const int y = i / E, e = i - y * E;
        double ax = 0.0, ay = 0.0;
        for (int k = 0; k < Ny; ++k) {
            const double d = D[y * Ny + k];
            const double2 x = v[(size_t)k * E + e];
            ax += d * x.x;
            ay += d * x.y;
        }
        o[i] = make_double2(ax, ay);
    }
}

// launch k = 0 .. E: CTAs 0 .. E-k-2 take x_{k+1+b} -= (<x_k, x_j> / <x_k, x_k>) x_k
// (v, eta and Dv); for k >= 1 the last CTA normalises x_{k-1} and records its
// norm (energy, the 1/4 included).
__global__ void __launch_bounds__(GS_THREADS) k_lin_gs(GroupView g, int k) {
    __shared__ double red[32];
    const int E = g.E, Ny = g.ny, NM = g.nmodes;
    const int nproj = k < E ? E - k - 1 : 0;
    const double* w = g.ccw + 1;
    double2* V = g.v_t;
    double2* H = g.e_t;
    double2* DV = g.v_s;
    const int n = NM * Ny;   // elements of one vector per field, H index (q Ny + y) E + member
    if ((int)blockIdx.x < nproj) {
        const int j = k + 1 + blockIdx.x;
        double nn = 0.0, cr = 0.0, ci = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int q = i / Ny, y = i - q * Ny;
            const double wy = w[y], wk = wy * g.k2inv[q];
            const size_t hk = (size_t)i * E + k, hj = (size_t)i * E + j;
            const double2 a0 = V[hk], b0 = V[hj], a1 = DV[hk], b1 = DV[hj], a2 = H[hk], b2 = H[hj];
            nn += wy * (a0.x * a0.x + a0.y * a0.y) + wk * (a1.x * a1.x + a1.y * a1.y + a2.x * a2.x + a2.y * a2.y);
            cr += wy * (a0.x * b0.x + a0.y * b0.y) + wk * (a1.x * b1.x + a1.y * b1.y + a2.x * b2.x + a2.y * b2.y);
            ci += wy * (a0.x * b0.y - a0.y * b0.x) + wk * (a1.x * b1.y - a1.y * b1.x + a2.x * b2.y - a2.y * b2.x);
        }
        nn = block_sum(nn, red);
        cr = block_sum(cr, red);
        ci = block_sum(ci, red);
        const double cx = cr / nn, cy = ci / nn;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const size_t hk = (size_t)i * E + k, hj = (size_t)i * E + j;
            double2* arr[3] = {V, DV, H};
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const double2 a = arr[f][hk];
                double2 b = arr[f][hj];
                b.x -= cx * a.x - cy * a.y;
                b.y -= cx * a.y + cy * a.x;
                arr[f][hj] = b;
            }
        }
    } else {
        const int j = k - 1;
        double nn = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int q = i / Ny, y = i - q * Ny;
            const double wy = w[y], wk = wy * g.k2inv[q];
            const size_t hj = (size_t)i * E + j;
            const double2 a0 = V[hj], a1 = DV[hj], a2 = H[hj];
            nn += wy * (a0.x * a0.x + a0.y * a0.y) + wk * (a1.x * a1.x + a1.y * a1.y + a2.x * a2.x + a2.y * a2.y);
        }
        nn = block_sum(nn, red);
        const double r = sqrt(0.25 * nn);
        if (threadIdx.x == 0) g.gsr[j] = r;
        const double s = 1.0 / r;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const size_t hj = (size_t)i * E + j;
            V[hj] = make_double2(V[hj].x * s, V[hj].y * s);
            H[hj] = make_double2(H[hj].x * s, H[hj].y * s);
        }
    }
}

int launch_lin_orthonormalize(const GroupView& g, cudaStream_t st) {
    k_lin_dv<<<g.nmodes, GS_THREADS, sizeof(double) * (size_t)g.ny * g.ny, st>>>(g);
    int launches = 1;
    for (int k = 0; k <= g.E; ++k) {
        const int nproj = k < g.E ? g.E - k - 1 : 0;
        const int grid = nproj + (k >= 1 ? 1 : 0);
        if (grid > 0) {
            k_lin_gs<<<grid, GS_THREADS, 0, st>>>(g, k);
            ++launches;
        }
    }
    return launches;
}

void set_attributes_linear() {
    allow_max_dynamic_smem(k_lin_dv);
    // the plane stage needs at most 2 x 9 x 128 x 16 B = 36 KB, below the default limit
}

}  // namespace dnsk
