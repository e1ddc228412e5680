// Single-precision physical-space stage (mixed path), one CTA per (interior
// y-plane, member).  Same mathematics as k_plane.cu (paper Sec. 3.1-3.2: u, w
// from v, eta; 12 inverse transforms with 2/3-rule zero padding; advective
// products N_i = u_j d_j u_i; plane means <uv>, <wv>; 3 forward transforms with
// truncation), organised for throughput:
//   * the five spectral inputs of the plane are staged in shared memory once;
//   * every length-N transform is a four-step N = N1 x N2 FFT: N2 tasks do
//     N1-point DFTs in registers, twiddle, exchange through shared memory once,
//     then N1 tasks do N2-point DFTs -- two barriers per 1-D stage;
//   * three fields (u, v, w, or the three derivatives of one component) are
//     transformed together, and the three derivative planes are folded into the
//     advective sum in one elementwise pass in a fixed order (deterministic).
#include "dns_internal.hpp"
#include "ff.cuh"

namespace dnsk {

namespace f32 {

template <int N> struct Split;
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct Split<48> { static constexpr int N1 = 6, N2 = 8; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// multiply by SIGN * i
template <int SIGN> __device__ __forceinline__ float2 mulsi(float2 a) {
    return SIGN > 0 ? f2(-a.y, a.x) : f2(a.y, -a.x);
}

// In-register DFTs, natural order in and out, kernel exp(SIGN 2 pi i jk / R).
template <int R, int SIGN> struct Dft;

template <int SIGN> struct Dft<2, SIGN> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = add(a, b); v[1] = sub(a, b);
    }
};
template <int SIGN> struct Dft<3, SIGN> {
    __device__ __forceinline__ static void run(float2* v) {
        const float h = 0.86602540378443864676f;   // sqrt(3)/2
        float2 t1 = add(v[1], v[2]), t2 = sub(v[1], v[2]);
        float2 x0 = add(v[0], t1);
        float2 m = f2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
        float2 s = mulsi<SIGN>(f2(h * t2.x, h * t2.y));
        v[0] = x0; v[1] = add(m, s); v[2] = sub(m, s);
    }
};
template <int SIGN> struct Dft<4, SIGN> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = add(v[0], v[2]), b = sub(v[0], v[2]);
        float2 c = add(v[1], v[3]), d = mulsi<SIGN>(sub(v[1], v[3]));
        v[0] = add(a, c); v[2] = sub(a, c);
        v[1] = add(b, d); v[3] = sub(b, d);
    }
};
// radix-2 decimation in time over two half-length DFTs
template <int SIGN> struct Dft<6, SIGN> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[3] = {v[0], v[2], v[4]}, o[3] = {v[1], v[3], v[5]};
        Dft<3, SIGN>::run(e);
        Dft<3, SIGN>::run(o);
        const float h = 0.86602540378443864676f;
        float2 w1 = f2(0.5f, SIGN * h), w2 = f2(-0.5f, SIGN * h);
        float2 t0 = o[0], t1 = mul(o[1], w1), t2 = mul(o[2], w2);
        v[0] = add(e[0], t0); v[3] = sub(e[0], t0);
        v[1] = add(e[1], t1); v[4] = sub(e[1], t1);
        v[2] = add(e[2], t2); v[5] = sub(e[2], t2);
    }
};
template <int SIGN> struct Dft<8, SIGN> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, SIGN>::run(e);
        Dft<4, SIGN>::run(o);
        const float c = 0.70710678118654752440f;
        float2 t0 = o[0];
        float2 t1 = mul(o[1], f2(c, SIGN * c));
        float2 t2 = mulsi<SIGN>(o[2]);
        float2 t3 = mul(o[3], f2(-c, SIGN * c));
        v[0] = add(e[0], t0); v[4] = sub(e[0], t0);
        v[1] = add(e[1], t1); v[5] = sub(e[1], t1);
        v[2] = add(e[2], t2); v[6] = sub(e[2], t2);
        v[3] = add(e[3], t3); v[7] = sub(e[3], t3);
    }
};

template <int MX, int MZ>
struct Cfg {
    static constexpr int KX = (MX - 1) / 3, KZ = (MZ - 1) / 3;
    static constexpr int NKX = KX + 1, NKZ = 2 * KZ + 1, NM = NKX * NKZ;
    static constexpr int NKXP = NKX | 1;          // odd row stride: conflict-free 8-byte columns
    static constexpr int X1 = Split<MX>::N1, X2 = Split<MX>::N2;
    static constexpr int Z1 = Split<MZ>::N1, Z2 = Split<MZ>::N2;
    static constexpr int HP = MZ / 2;             // line pairs of the x transforms
    static constexpr int PLANE = MX * MZ;
    static constexpr int NF = 3;                  // fields transformed together
    // Layouts (consecutive threads always touch consecutive words):
    //   physical planes [x][z];  A (z-transformed columns) [z][n] stride NKXP;
    //   z exchange [k1][n2][n] stride NKXP;  x exchange [k1][n2][p];  x output [x][p]
    static constexpr int SZ = Z1 * Z2 * NKXP;
    static constexpr int SX = X1 * X2 * HP;
    static constexpr int SSP = SZ > SX ? SZ : SX;   // = also MX * HP (one output plane)
    static constexpr int AS = MZ * NKXP;
    static constexpr int NT0 = NF * HP * X2;
    static constexpr int NT = ((NT0 + 31) / 32) * 32 > 1024 ? 1024 : ((NT0 + 31) / 32) * 32;
    // shared-memory layout (bytes)
    static constexpr size_t B_BASE = 0;                                   // float2 [5][NM]
    static constexpr size_t B_PLN = B_BASE + sizeof(float2) * 5 * NM;     // float  [3][PLANE]: u, v, w
    static constexpr size_t B_A = B_PLN + sizeof(float) * 3 * PLANE;      // float2 [2 NF][AS]: working + u, v, w
    static constexpr size_t B_S = B_A + sizeof(float2) * 2 * NF * AS;     // float2 [NF][SSP]
    static constexpr size_t B_TW = B_S + sizeof(float2) * NF * SSP;       // float2 [MX + MZ]
    static constexpr size_t B_K = B_TW + sizeof(float2) * (MX + MZ);      // float [NKX + NKZ + NM]
    static constexpr size_t B_RED = ((B_K + sizeof(float) * (NKX + NKZ + NM)) + 15) / 16 * 16;
    static constexpr size_t BYTES = B_RED + 64 * sizeof(double);
};

template <int MX, int MZ>
__global__ void __launch_bounds__(Cfg<MX, MZ>::NT, 1)
k_plane_f32(GroupView g, const double* __restrict__ Ucur, const double* __restrict__ Wcur) {
    typedef Cfg<MX, MZ> K;
    constexpr int KX = K::KX, KZ = K::KZ, NKX = K::NKX, NM = K::NM;
    constexpr int X1 = K::X1, X2 = K::X2, Z1 = K::Z1, Z2 = K::Z2, HP = K::HP, PLANE = K::PLANE;
    constexpr int NF = K::NF;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* base = (float2*)(smem + K::B_BASE);
    float* pl = (float*)(smem + K::B_PLN);
    float* PU = pl;
    float* PV = pl + PLANE;
    float* PW = pl + 2 * PLANE;
    float2* Ab = (float2*)(smem + K::B_A);
    float2* Sb = (float2*)(smem + K::B_S);
    float2* twx = (float2*)(smem + K::B_TW);
    float2* twz = twx + MX;
    float* kxs = (float*)(smem + K::B_K);
    float* kzs = kxs + NKX;
    float* k2s = kzs + K::NKZ;
    double* red = (double*)(smem + K::B_RED);

    const int tid = threadIdx.x;
    constexpr int NT = K::NT;
    const int y = blockIdx.x, e = blockIdx.y, E = g.E, Ny = g.ny, My = g.my;
    const size_t fs = (size_t)Ny * E * NM;
    const size_t off0 = ((size_t)y * E + e) * NM;

    // ---- stage inputs and tables
    {
        const float2* P = (const float2*)g.P5;
        for (int i = tid; i < 5 * NM; i += NT) {
            int f = i / NM, q = i - f * NM;
            base[i] = P[f * fs + off0 + q];
        }
        for (int i = tid; i < MX; i += NT) twx[i] = g.twxf[i];
        for (int i = tid; i < MZ; i += NT) twz[i] = g.twzf[i];
        for (int i = tid; i < NKX; i += NT) kxs[i] = g.kxtf[i];
        for (int i = tid; i < K::NKZ; i += NT) kzs[i] = g.kztf[i];
        for (int i = tid; i < NM; i += NT) k2s[i] = g.k2invf[i];
    }
    const float Um = (float)Ucur[(size_t)e * My + y + 1];
    const float Wm = (float)Wcur[(size_t)e * My + y + 1];
    mean_dy_row(g.D1, Ucur + (size_t)e * My, Wcur + (size_t)e * My, My, y + 1, red);
    const float2* Bv = base;
    const float2* BDv = base + NM;
    const float2* BD2v = base + 2 * NM;
    const float2* Be = base + 3 * NM;
    const float2* BDe = base + 4 * NM;
    constexpr int QMEAN = KZ * NKX;
    __syncthreads();
    const float dUm = (float)red[0];
    const float dWm = (float)red[1];
    __syncthreads();

    // spectral value of field `which` at mode (mi, n): 0 u, 1 v, 2 w,
    // 3 + 3 i + j = d u_i / d x_j
    auto gen = [&](int which, int mi, int n) -> float2 {
        const int q = mi * NKX + n;
        const float kx = kxs[n], kz = kzs[mi], ki = k2s[q];
        const bool mean = (q == QMEAN);
        const int comp = which < 3 ? which : (which - 3) / 3;
        const int dir = which < 3 ? -1 : (which - 3) % 3;
        if (dir == 1) {
            if (comp == 1) return BDv[q];
            if (mean) return f2(comp == 0 ? dUm : dWm, 0.f);
            float2 d2 = BD2v[q], de = BDe[q];
            float ax, ay;
            if (comp == 0) { ax = (kx * d2.x - kz * de.x) * ki; ay = (kx * d2.y - kz * de.y) * ki; }
            else { ax = (kz * d2.x + kx * de.x) * ki; ay = (kz * d2.y + kx * de.y) * ki; }
            return f2(-ay, ax);
        }
        float2 b;
        if (comp == 1) {
            b = Bv[q];
        } else if (mean) {
            b = f2(comp == 0 ? Um : Wm, 0.f);
        } else {
            float2 dv = BDv[q], et = Be[q];
            float ax, ay;
            if (comp == 0) { ax = (kx * dv.x - kz * et.x) * ki; ay = (kx * dv.y - kz * et.y) * ki; }
            else { ax = (kz * dv.x + kx * et.x) * ki; ay = (kz * dv.y + kx * et.y) * ki; }
            b = f2(-ay, ax);
        }
        if (dir < 0) return b;
        const float k = dir == 0 ? kx : kz;
        return f2(-k * b.y, k * b.x);
    };

    // ---- inverse transforms of three fields; mode 0 (u, v, w): into PU/PV/PW,
    // their z-transformed columns kept in A slots 3..5; mode 1 (the three
    // derivatives of component xc): into the per-field scratch as [x][p]
    // line-pair planes.  The x derivative needs no z-stage of its own: the
    // z transform commutes with the factor i kx, so its x-stage reads the
    // kept columns of u_xc times i kx.
    constexpr int NKXP = K::NKXP, AS = K::AS, SSP = K::SSP;
    auto inverse3 = [&](int w0, int w1, int w2, int mode, int xc) {
        const int f_lo = (mode == 1) ? 1 : 0;      // the x derivative skips the z-stage
        auto aslot = [&](int f) -> float2* { return Ab + (mode == 0 ? 3 + f : f) * AS; };
        // z-stage, step A: tasks (f, n2, n), n fastest
        for (int t = tid; t < (NF - f_lo) * NKX * Z2; t += NT) {
            const int n = t % NKX, r = t / NKX, n2 = r % Z2, f = f_lo + r / Z2;
            const int which = f == 0 ? w0 : (f == 1 ? w1 : w2);
            float2 v[Z1];
#pragma unroll
            for (int n1 = 0; n1 < Z1; ++n1) {
                const int z = Z2 * n1 + n2;
                int mi = -1;
                if (z <= KZ) mi = z + KZ;
                else if (z >= MZ - KZ) mi = z - MZ + KZ;
                v[n1] = mi >= 0 ? gen(which, mi, n) : f2(0.f, 0.f);
            }
            Dft<Z1, +1>::run(v);
            float2* S = Sb + f * SSP + n2 * NKXP + n;
#pragma unroll
            for (int k1 = 0; k1 < Z1; ++k1) {
                float2 w = twz[n2 * k1];
                S[k1 * (Z2 * NKXP)] = k1 == 0 ? v[0] : mul(v[k1], f2(w.x, -w.y));
            }
        }
        __syncthreads();
        // z-stage, step C: tasks (f, k1, n) -> A[f][z][n]
        for (int t = tid; t < (NF - f_lo) * NKX * Z1; t += NT) {
            const int n = t % NKX, r = t / NKX, k1 = r % Z1, f = f_lo + r / Z1;
            const float2* S = Sb + f * SSP + k1 * (Z2 * NKXP) + n;
            float2 v[Z2];
#pragma unroll
            for (int n2 = 0; n2 < Z2; ++n2) v[n2] = S[n2 * NKXP];
            Dft<Z2, +1>::run(v);
            float2* A = aslot(f) + n;
#pragma unroll
            for (int k2 = 0; k2 < Z2; ++k2) A[(k1 + Z1 * k2) * NKXP] = v[k2];
        }
        __syncthreads();
        // x-stage, step A: tasks (f, n2, p), p fastest; line p carries rows p, p + HP
        for (int t = tid; t < NF * HP * X2; t += NT) {
            const int p = t % HP, r = t / HP, n2 = r % X2, f = r / X2;
            const bool dx = (f == 0 && mode == 1);          // x derivative of u_xc
            const float2* A0 = (dx ? Ab + (3 + xc) * AS : aslot(f)) + p * NKXP;
            const float2* A1 = A0 + HP * NKXP;
            float2 v[X1];
#pragma unroll
            for (int n1 = 0; n1 < X1; ++n1) {
                const int k = X2 * n1 + n2;
                float2 Z = f2(0.f, 0.f);
                if (k == 0) {
                    if (!dx) Z = f2(A0[0].x, A1[0].x);        // Hermitian part of the n = 0 column
                } else if (k <= KX) {
                    float2 a = A0[k], b = A1[k];
                    if (dx) { const float kx = kxs[k]; a = f2(-kx * a.y, kx * a.x); b = f2(-kx * b.y, kx * b.x); }
                    Z = f2(a.x - b.y, a.y + b.x);             // a + i b
                } else if (k >= MX - KX) {
                    float2 a = A0[MX - k], b = A1[MX - k];
                    if (dx) { const float kx = kxs[MX - k]; a = f2(-kx * a.y, kx * a.x); b = f2(-kx * b.y, kx * b.x); }
                    Z = f2(a.x + b.y, b.x - a.y);             // conj(a) + i conj(b)
                }
                v[n1] = Z;
            }
            Dft<X1, +1>::run(v);
            float2* S = Sb + f * SSP + n2 * HP + p;
#pragma unroll
            for (int k1 = 0; k1 < X1; ++k1) {
                float2 w = twx[n2 * k1];
                S[k1 * (X2 * HP)] = k1 == 0 ? v[0] : mul(v[k1], f2(w.x, -w.y));
            }
        }
        __syncthreads();
        // x-stage, step C: one task (f, k1, p) per thread
        static_assert(NF * HP * X1 <= NT, "one x-stage step-C task per thread");
        float2 out[X2];
        const bool active = tid < NF * HP * X1;
        int cf = 0, cp = 0, ck1 = 0;
        if (active) {
            cp = tid % HP;
            const int r = tid / HP;
            ck1 = r % X1;
            cf = r / X1;
            const float2* S = Sb + cf * SSP + ck1 * (X2 * HP) + cp;
#pragma unroll
            for (int n2 = 0; n2 < X2; ++n2) out[n2] = S[n2 * HP];
            Dft<X2, +1>::run(out);
        }
        if (mode == 1) __syncthreads();     // the scratch is overwritten below
        if (active) {
            if (mode == 0) {
                float* dst = pl + cf * PLANE + cp;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) {
                    const int x = ck1 + X1 * k2;
                    dst[x * MZ] = out[k2].x;
                    dst[x * MZ + HP] = out[k2].y;
                }
            } else {
                float2* dst = Sb + cf * SSP + cp;
#pragma unroll
                for (int k2 = 0; k2 < X2; ++k2) dst[(ck1 + X1 * k2) * HP] = out[k2];
            }
        }
        __syncthreads();
    };

    // ---- forward transform of the advective sum, held in slot 0 as packed
    // line pairs [x][p] (row p in .x, row p + HP in .y); kept modes to global
    auto forward = [&](float2* __restrict__ gout) {
        // x-stage, step A: tasks (n2, p), p fastest; exchange in slot 1
        for (int t = tid; t < HP * X2; t += NT) {
            const int p = t % HP, n2 = t / HP;
            float2 v[X1];
#pragma unroll
            for (int n1 = 0; n1 < X1; ++n1) v[n1] = Sb[(X2 * n1 + n2) * HP + p];
            Dft<X1, -1>::run(v);
            float2* S = Sb + SSP + n2 * HP + p;
#pragma unroll
            for (int k1 = 0; k1 < X1; ++k1) S[k1 * (X2 * HP)] = k1 == 0 ? v[0] : mul(v[k1], twx[n2 * k1]);
        }
        __syncthreads();
        // x-stage, step C: tasks (k1, p), outputs [x][p] into slot 2
        for (int t = tid; t < HP * X1; t += NT) {
            const int p = t % HP, k1 = t / HP;
            const float2* S = Sb + SSP + k1 * (X2 * HP) + p;
            float2 v[X2];
#pragma unroll
            for (int n2 = 0; n2 < X2; ++n2) v[n2] = S[n2 * HP];
            Dft<X2, -1>::run(v);
            float2* O = Sb + 2 * SSP + p;
#pragma unroll
            for (int k2 = 0; k2 < X2; ++k2) O[(k1 + X1 * k2) * HP] = v[k2];
        }
        __syncthreads();
        // split the two real rows, keep n <= KX, scale 1/MX -> A[0][z][n]
        const float sx = 1.0f / MX;
        for (int t = tid; t < HP * NKX; t += NT) {
            const int p = t % HP, n = t / HP;
            const float2* O = Sb + 2 * SSP + p;
            float2 Zn = O[n * HP], Zc = O[((MX - n) % MX) * HP];
            float2 xa = f2(0.5f * (Zn.x + Zc.x) * sx, 0.5f * (Zn.y - Zc.y) * sx);
            float2 xb = f2(0.5f * (Zn.y + Zc.y) * sx, 0.5f * (Zc.x - Zn.x) * sx);
            Ab[p * NKXP + n] = xa;
            Ab[(p + HP) * NKXP + n] = xb;
        }
        __syncthreads();
        // z-stage, step A: tasks (n2, n), n fastest
        for (int t = tid; t < NKX * Z2; t += NT) {
            const int n = t % NKX, n2 = t / NKX;
            float2 v[Z1];
#pragma unroll
            for (int n1 = 0; n1 < Z1; ++n1) v[n1] = Ab[(Z2 * n1 + n2) * NKXP + n];
            Dft<Z1, -1>::run(v);
            float2* S = Sb + n2 * NKXP + n;
#pragma unroll
            for (int k1 = 0; k1 < Z1; ++k1) S[k1 * (Z2 * NKXP)] = k1 == 0 ? v[0] : mul(v[k1], twz[n2 * k1]);
        }
        __syncthreads();
        // z-stage, step C: tasks (k1, n); keep |m| <= KZ, scale 1/MZ -> staging [NM]
        float2* stage = Sb + SSP;
        const float sz = 1.0f / MZ;
        for (int t = tid; t < NKX * Z1; t += NT) {
            const int n = t % NKX, k1 = t / NKX;
            const float2* S = Sb + k1 * (Z2 * NKXP) + n;
            float2 v[Z2];
#pragma unroll
            for (int n2 = 0; n2 < Z2; ++n2) v[n2] = S[n2 * NKXP];
            Dft<Z2, -1>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < Z2; ++k2) {
                const int m = k1 + Z1 * k2;
                int mi = -1;
                if (m <= KZ) mi = m + KZ;
                else if (m >= MZ - KZ) mi = m - MZ + KZ;
                if (mi >= 0) stage[mi * NKX + n] = f2(v[k2].x * sz, v[k2].y * sz);
            }
        }
        __syncthreads();
        for (int i = tid; i < NM; i += NT) gout[i] = stage[i];
        __syncthreads();
    };

    // velocities
    inverse3(0, 1, 2, 0, -1);
    // plane means <uv>, <wv>
    {
        // float-float sums (the FP64 pipe is slow)
        float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int i = tid; i < PLANE; i += NT) {
            ff_add_prod(h1, l1, PU[i], PV[i]);
            ff_add_prod(h2, l2, PW[i], PV[i]);
        }
        double s1 = 0.0, s2 = 0.0;
        ff_block_sum2(h1, l1, h2, l2, (float*)red, &s1, &s2);
        if (tid == 0) {
            g.uv[(size_t)e * My + y + 1] = s1 / (double)PLANE;
            g.wv[(size_t)e * My + y + 1] = s2 / (double)PLANE;
        }
    }
    float2* N3 = (float2*)g.N3;
    for (int i = 0; i < 3; ++i) {
        inverse3(3 + 3 * i, 4 + 3 * i, 5 + 3 * i, 1, i);
        // N_i = u d_x u_i + v d_y u_i + w d_z u_i, in this order, written over
        // the d_x plane in the same packed line-pair form
        float2* G0 = Sb;
        const float2* G1 = Sb + SSP;
        const float2* G2 = Sb + 2 * SSP;
        for (int t = tid; t < HP * MX; t += NT) {
            const int p = t % HP, x = t / HP;
            const float2 a = G0[t], b = G1[t], c = G2[t];
            const int i0 = x * MZ + p, i1 = i0 + HP;
            G0[t] = f2(PU[i0] * a.x + PV[i0] * b.x + PW[i0] * c.x, PU[i1] * a.y + PV[i1] * b.y + PW[i1] * c.y);
        }
        __syncthreads();
        forward(N3 + (size_t)i * fs + off0);
    }
}

template <int MX, int MZ>
void launch_t(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
    typedef Cfg<MX, MZ> K;
    k_plane_f32<MX, MZ><<<dim3(g.ny, g.E), K::NT, K::BYTES, st>>>(g, U, W);
}

template <int MX, int MZ>
void set_attr_t() {
    typedef Cfg<MX, MZ> K;
    static_assert(K::BYTES <= 227 * 1024, "plane stage does not fit in shared memory");
    cudaFuncSetAttribute(k_plane_f32<MX, MZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::BYTES);
}

}  // namespace f32

#define DNS_PLANE_SIZES(X) X(16, 16) X(16, 32) X(16, 48) X(16, 64) X(32, 16) X(32, 32) X(32, 48) X(32, 64) \
    X(48, 16) X(48, 32) X(48, 48) X(48, 64) X(64, 16) X(64, 32) X(64, 48) X(64, 64)

bool launch_plane_f32(const GroupView& g, const double* U, const double* W, cudaStream_t st) {
#define DNS_CASE(a, b) if (g.mx == a && g.mz == b) { f32::launch_t<a, b>(g, U, W, st); return true; }
    DNS_PLANE_SIZES(DNS_CASE)
#undef DNS_CASE
    return false;
}

size_t plane_f32_smem_bytes(int mx, int mz) {
#define DNS_CASE(a, b) if (mx == a && mz == b) return f32::Cfg<a, b>::BYTES;
    DNS_PLANE_SIZES(DNS_CASE)
#undef DNS_CASE
    return 0;
}

void set_attributes_plane_f32() {
#define DNS_CASE(a, b) f32::set_attr_t<a, b>();
    DNS_PLANE_SIZES(DNS_CASE)
#undef DNS_CASE
}

}  // namespace dnsk
