// Four-step FFT building blocks shared by the plane-stage kernels: complex
// helpers generic in the component type, in-register DFTs of the radices the
// supported grid sizes need (natural order in and out), and the N = N1 x N2
// factorisation used for each transform length.
#pragma once
#include <cuda_runtime.h>

namespace dnsk {
namespace dft {

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

template <typename C, typename T>
__device__ __forceinline__ C mk(T a, T b) { C r; r.x = a; r.y = b; return r; }
template <typename C>
__device__ __forceinline__ C add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C mul(C a, C b) { C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; }
template <int SIGN, typename C>
__device__ __forceinline__ C mulsi(C a) { C r; if (SIGN > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r; }
template <typename C, typename T>
__device__ __forceinline__ C scal(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }

// In-register DFTs, natural order in and out, kernel exp(SIGN 2 pi i jk / R).
template <int R, int SIGN, typename C> struct Dft;
template <int SIGN, typename C> struct Dft<3, SIGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(v[0].x) T;
        const T h = (T)0.86602540378443864676;
        C t1 = add(v[1], v[2]), t2 = sub(v[1], v[2]);
        C x0 = add(v[0], t1);
        C m = mk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        C s = mulsi<SIGN>(scal(t2, h));
        v[0] = x0; v[1] = add(m, s); v[2] = sub(m, s);
    }
};
template <int SIGN, typename C> struct Dft<4, SIGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        C a = add(v[0], v[2]), b = sub(v[0], v[2]);
        C c = add(v[1], v[3]), d = mulsi<SIGN>(sub(v[1], v[3]));
        v[0] = add(a, c); v[2] = sub(a, c);
        v[1] = add(b, d); v[3] = sub(b, d);
    }
};
template <int SIGN, typename C> struct Dft<6, SIGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(v[0].x) T;
        C e[3] = {v[0], v[2], v[4]}, o[3] = {v[1], v[3], v[5]};
        Dft<3, SIGN, C>::run(e);
        Dft<3, SIGN, C>::run(o);
        const T h = (T)0.86602540378443864676;
        C t0 = o[0], t1 = mul(o[1], mk<C>((T)0.5, (T)SIGN * h)), t2 = mul(o[2], mk<C>((T)-0.5, (T)SIGN * h));
        v[0] = add(e[0], t0); v[3] = sub(e[0], t0);
        v[1] = add(e[1], t1); v[4] = sub(e[1], t1);
        v[2] = add(e[2], t2); v[5] = sub(e[2], t2);
    }
};
template <int SIGN, typename C> struct Dft<8, SIGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(v[0].x) T;
        C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, SIGN, C>::run(e);
        Dft<4, SIGN, C>::run(o);
        const T c = (T)0.70710678118654752440;
        C t0 = o[0], t1 = mul(o[1], mk<C>(c, (T)SIGN * c)), t2 = mulsi<SIGN>(o[2]), t3 = mul(o[3], mk<C>(-c, (T)SIGN * c));
        v[0] = add(e[0], t0); v[4] = sub(e[0], t0);
        v[1] = add(e[1], t1); v[5] = sub(e[1], t1);
        v[2] = add(e[2], t2); v[6] = sub(e[2], t2);
        v[3] = add(e[3], t3); v[7] = sub(e[3], t3);
    }
};
template <int SIGN, typename C> struct Dft<16, SIGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(v[0].x) T;
        C e[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
        Dft<8, SIGN, C>::run(e);
        Dft<8, SIGN, C>::run(o);
        const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, c2 = (T)0.70710678118654752440;
        const T S = (T)SIGN;
        const C w[8] = {mk<C>((T)1, (T)0), mk<C>(c1, S * s1), mk<C>(c2, S * c2), mk<C>(s1, S * c1),
                        mk<C>((T)0, S), mk<C>(-s1, S * c1), mk<C>(-c2, S * c2), mk<C>(-c1, S * s1)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            C t = k == 0 ? o[0] : mul(o[k], w[k]);
            v[k] = add(e[k], t);
            v[k + 8] = sub(e[k], t);
        }
    }
};

template <int N> struct Split;
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct Split<48> { static constexpr int N1 = 6, N2 = 8; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 8, N2 = 16; };

constexpr int cmax(int a, int b) { return a > b ? a : b; }

}  // namespace dft
}  // namespace dnsk
