// Physical-space stage of one sub-step (paper Sec. 3.1 and 3.2): for one
// interior y-plane of one member,
//   1. synthesise u, v, w and their nine first derivatives in spectral space
//      from v, Dv, D2v, eta, D eta (u = i(kx Dv - kz eta)/k^2,
//      w = i(kz Dv + kx eta)/k^2, x/z derivatives as i kx, i kz factors, the
//      (0,0) mode carrying U00, W00 and their y-derivatives),
//   2. inverse-transform each to the Mx x Mz grid (zero-padded, 2/3 rule),
//   3. form the advective products N_i = u du_i/dx + v du_i/dy + w du_i/dz and
//      the plane means <uv>, <wv>,
//   4. forward-transform N_u, N_v, N_w and keep |n| <= Kx, |m| <= Kz.
// Transforms: z first (c2c over the kept n columns), then x (two real rows
// packed as one complex line).  Everything stays in shared memory; the only
// global traffic is the 5 spectral inputs and 3 spectral outputs per plane.
#include "dns_internal.hpp"
#include <climits>

namespace dnsk {

constexpr int PLANE_THREADS = 256;
constexpr int CHUNK = 16;   // FFT lines processed per batch

int plane_threads() { return PLANE_THREADS; }

size_t plane_smem_bytes(const GroupView& g, int eb) {
    size_t cb = 2 * (size_t)eb;
    size_t plane = (size_t)g.mx * g.mz;
    int lmax = g.mx > g.mz ? g.mx : g.mz;
    size_t b = 4 * plane * eb;
    b += ((size_t)g.nkx * g.mz + 2 * (size_t)CHUNK * lmax + g.mx + g.mz) * cb;
    b += 32 * sizeof(double);
    return b;
}

template <typename T>
__global__ void __launch_bounds__(PLANE_THREADS) k_plane(GroupView g, const double* __restrict__ Ucur,
                                                         const double* __restrict__ Wcur) {
    typedef typename C2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Mx = g.mx, Mz = g.mz, NKX = g.nkx, Kx = g.kx, Kz = g.kz, nmodes = g.nmodes;
    const int y = blockIdx.x, e = blockIdx.y, E = g.E, Ny = g.ny, My = g.my;
    const int plane = Mx * Mz;
    const int half = Mz / 2;
    const int lmax = Mx > Mz ? Mx : Mz;
    const int tid = threadIdx.x, nthr = blockDim.x;

    T* PU = (T*)smem;
    T* PV = PU + plane;
    T* PW = PV + plane;
    T* ACC = PW + plane;
    C* A = (C*)(ACC + plane);
    C* W0 = A + NKX * Mz;
    C* W1 = W0 + CHUNK * lmax;
    C* twx = W1 + CHUNK * lmax;
    C* twz = twx + Mx;
    double* red = (double*)(twz + Mz);

    const C* twxg = (const C*)(sizeof(T) == 8 ? (const void*)g.twx : (const void*)g.twxf);
    const C* twzg = (const C*)(sizeof(T) == 8 ? (const void*)g.twz : (const void*)g.twzf);
    for (int i = tid; i < Mx; i += nthr) twx[i] = twxg[i];
    for (int i = tid; i < Mz; i += nthr) twz[i] = twzg[i];

    const C* P = (const C*)g.P5;
    const size_t fs = (size_t)Ny * E * nmodes;
    const size_t off0 = ((size_t)y * E + e) * nmodes;
    const C* Pv = P + off0;
    const C* PDv = P + fs + off0;
    const C* PD2v = P + 2 * fs + off0;
    const C* Pe = P + 3 * fs + off0;
    const C* PDe = P + 4 * fs + off0;
    const T* kxt = (const T*)(sizeof(T) == 8 ? (const void*)g.kxt : (const void*)g.kxtf);
    const T* kzt = (const T*)(sizeof(T) == 8 ? (const void*)g.kzt : (const void*)g.kztf);
    const T* k2i = (const T*)(sizeof(T) == 8 ? (const void*)g.k2inv : (const void*)g.k2invf);
    const int q_mean = Kz * NKX;
    const T Um = (T)Ucur[(size_t)e * My + y + 1];
    const T Wm = (T)Wcur[(size_t)e * My + y + 1];
    mean_dy_row(g.D1, Ucur + (size_t)e * My, Wcur + (size_t)e * My, My, y + 1, red);
    __syncthreads();
    const T dUm = (T)red[0];
    const T dWm = (T)red[1];
    __syncthreads();

    // spectral value of field `which` at mode q:
    //   0 u, 1 v, 2 w, 3 + 3 i + j: d u_i / d x_j (i: u v w, j: x y z),
    //   12, 13, 14: vorticity omega_x = dw/dy - dv/dz, omega_y = eta,
    //   omega_z = dv/dx - du/dy
    auto gen0 = [&](int which, int q) -> C {
        const int mi = q / NKX, n = q - mi * NKX;
        const T kx = kxt[n], kz = kzt[mi], ki = k2i[q];
        const bool mean = (q == q_mean);
        int comp = which < 3 ? which : (which - 3) / 3;
        int dir = which < 3 ? -1 : (which - 3) % 3;
        C r;
        if (dir == 1) {   // y-derivatives
            if (comp == 1) return PDv[q];
            if (mean) { r.x = comp == 0 ? dUm : dWm; r.y = 0; return r; }
            C d2 = PD2v[q], de = PDe[q];
            T ax, ay;
            if (comp == 0) { ax = (kx * d2.x - kz * de.x) * ki; ay = (kx * d2.y - kz * de.y) * ki; }
            else { ax = (kz * d2.x + kx * de.x) * ki; ay = (kz * d2.y + kx * de.y) * ki; }
            r.x = -ay; r.y = ax;
            return r;
        }
        C base;
        if (comp == 1) {
            base = Pv[q];
        } else if (mean) {
            base.x = comp == 0 ? Um : Wm; base.y = 0;
        } else {
            C dv = PDv[q], et = Pe[q];
            T ax, ay;
            if (comp == 0) { ax = (kx * dv.x - kz * et.x) * ki; ay = (kx * dv.y - kz * et.y) * ki; }
            else { ax = (kz * dv.x + kx * et.x) * ki; ay = (kz * dv.y + kx * et.y) * ki; }
            base.x = -ay; base.y = ax;
        }
        if (dir < 0) return base;
        T k = dir == 0 ? kx : kz;
        r.x = -k * base.y; r.y = k * base.x;
        return r;
    };
    auto genw = [&](int which, int q) -> C {
        if (which < 12) return gen0(which, q);
        if (which == 13) return Pe[q];
        C a = gen0(which == 12 ? 10 : 6, q), b = gen0(which == 12 ? 8 : 4, q);   // (wy - vz) or (vx - uy)
        a.x -= b.x; a.y -= b.y;
        return a;
    };

    // inverse transform of field `which`; acc = false: dst = field,
    // acc = true: dst += sgn vel * field
    auto inverse2d = [&](int which, bool acc, T* dst, const T* vel, T sgn) {
        for (int c0 = 0; c0 < NKX; c0 += CHUNK) {
            int nl = min(CHUNK, NKX - c0);
            for (int idx = tid; idx < nl * Mz; idx += nthr) {
                int l = idx / Mz, z = idx - l * Mz;
                int m = (z <= Kz) ? z : (z >= Mz - Kz ? z - Mz : INT_MIN);
                C val = czero<C>();
                if (m != INT_MIN) val = genw(which, (m + Kz) * NKX + c0 + l);
                W0[idx] = val;
            }
            __syncthreads();
            C* r = fft_lines<C, +1>(W0, W1, nl, g.pz, twz);
            for (int idx = tid; idx < nl * Mz; idx += nthr) A[c0 * Mz + idx] = r[idx];
            __syncthreads();
        }
        for (int p0 = 0; p0 < half; p0 += CHUNK) {
            int np = min(CHUNK, half - p0);
            for (int idx = tid; idx < np * Mx; idx += nthr) {
                int l = idx / Mx, k = idx - l * Mx;
                int z = p0 + l, z2 = z + half;
                C Z = czero<C>();
                if (k == 0) {
                    Z.x = A[z].x; Z.y = A[z2].x;
                } else if (k <= Kx) {
                    C a = A[k * Mz + z], b = A[k * Mz + z2];
                    Z.x = a.x - b.y; Z.y = a.y + b.x;
                } else if (k >= Mx - Kx) {
                    int n = Mx - k;
                    C a = A[n * Mz + z], b = A[n * Mz + z2];
                    Z.x = a.x + b.y; Z.y = b.x - a.y;
                }
                W0[idx] = Z;
            }
            __syncthreads();
            C* r = fft_lines<C, +1>(W0, W1, np, g.px, twx);
            for (int idx = tid; idx < np * Mx; idx += nthr) {
                int l = idx / Mx, x = idx - l * Mx;
                int z = p0 + l, z2 = z + half;
                C val = r[idx];
                if (!acc) {
                    dst[z * Mx + x] = val.x;
                    dst[z2 * Mx + x] = val.y;
                } else {
                    dst[z * Mx + x] += sgn * vel[z * Mx + x] * val.x;
                    dst[z2 * Mx + x] += sgn * vel[z2 * Mx + x] * val.y;
                }
            }
            __syncthreads();
        }
    };

    // forward transform of the real plane src, kept modes written to out[q]
    auto forward2d = [&](const T* src, C* out) {
        const T sx = (T)1 / (T)Mx, sz = (T)1 / (T)Mz;
        for (int p0 = 0; p0 < half; p0 += CHUNK) {
            int np = min(CHUNK, half - p0);
            for (int idx = tid; idx < np * Mx; idx += nthr) {
                int l = idx / Mx, x = idx - l * Mx;
                int z = p0 + l, z2 = z + half;
                C Z; Z.x = src[z * Mx + x]; Z.y = src[z2 * Mx + x];
                W0[idx] = Z;
            }
            __syncthreads();
            C* r = fft_lines<C, -1>(W0, W1, np, g.px, twx);
            for (int idx = tid; idx < np * (Kx + 1); idx += nthr) {
                int l = idx / (Kx + 1), n = idx - l * (Kx + 1);
                int z = p0 + l, z2 = z + half;
                C Zn = r[l * Mx + n];
                C Zc = r[l * Mx + ((Mx - n) % Mx)];
                // two real rows: Xa = (Zn + conj Zc)/2, Xb = (Zn - conj Zc)/(2i)
                C xa, xb;
                xa.x = (T)0.5 * (Zn.x + Zc.x) * sx; xa.y = (T)0.5 * (Zn.y - Zc.y) * sx;
                xb.x = (T)0.5 * (Zn.y + Zc.y) * sx; xb.y = (T)0.5 * (Zc.x - Zn.x) * sx;
                A[n * Mz + z] = xa;
                A[n * Mz + z2] = xb;
            }
            __syncthreads();
        }
        for (int c0 = 0; c0 < NKX; c0 += CHUNK) {
            int nl = min(CHUNK, NKX - c0);
            for (int idx = tid; idx < nl * Mz; idx += nthr) W0[idx] = A[c0 * Mz + idx];
            __syncthreads();
            C* r = fft_lines<C, -1>(W0, W1, nl, g.pz, twz);
            const int nkz = 2 * Kz + 1;
            for (int idx = tid; idx < nl * nkz; idx += nthr) {
                int mi = idx / nl, l = idx - mi * nl;
                int m = mi - Kz;
                int zz = m < 0 ? m + Mz : m;
                C v = r[l * Mz + zz];
                v.x *= sz; v.y *= sz;
                out[mi * NKX + c0 + l] = v;
            }
            __syncthreads();
        }
    };

    __syncthreads();
    inverse2d(0, false, PU, nullptr, (T)1);
    inverse2d(1, false, PV, nullptr, (T)1);
    inverse2d(2, false, PW, nullptr, (T)1);

    // plane means <uv>, <wv> (the (0,0) Fourier coefficients of the products)
    {
        double s1 = 0.0, s2 = 0.0;
        for (int i = tid; i < plane; i += nthr) {
            s1 += (double)PU[i] * (double)PV[i];
            s2 += (double)PW[i] * (double)PV[i];
        }
        s1 = block_sum(s1, red);
        s2 = block_sum(s2, red);
        if (tid == 0) {
            g.uv[(size_t)e * My + y + 1] = s1 / (double)plane;
            g.wv[(size_t)e * My + y + 1] = s2 / (double)plane;
        }
    }

    C* N3 = (C*)g.N3;
    const T* vel[3] = {PU, PV, PW};
    for (int i = 0; i < 3; ++i) {
        for (int k = tid; k < plane; k += nthr) ACC[k] = (T)0;
        __syncthreads();
        if (g.rot) {
            // rotational form N = omega x u: N_i = u_a omega_b - u_b omega_a,
            // (a, b) = (z, y) for i = x, (x, z) for y, (y, x) for z
            const int a = (i + 2) % 3, b = (i + 1) % 3;
            inverse2d(12 + b, true, ACC, vel[a], (T)1);
            inverse2d(12 + a, true, ACC, vel[b], (T)-1);
        } else {
            for (int j = 0; j < 3; ++j) inverse2d(3 + 3 * i + j, true, ACC, vel[j], (T)1);
        }
        forward2d(ACC, N3 + (size_t)i * fs + off0);
    }
}

template <typename T>
void launch_plane_state(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
    size_t smem = plane_smem_bytes(g, sizeof(T));
    k_plane<T><<<dim3(g.ny, g.E), PLANE_THREADS, smem, st>>>(g, U, W);
}
template void launch_plane_state<double>(const GroupView&, const double*, const double*, cudaStream_t);

void set_attributes_plane() {
    allow_max_dynamic_smem(k_plane<double>);
}

}  // namespace dnsk
