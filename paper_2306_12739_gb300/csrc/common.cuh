// Device-side helpers shared by the DNS kernels: complex arithmetic and the
// CTA-wide shared-memory FFT (Stockham autosort, mixed radix 2/3/4).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dnsk {

// Bounds checks of the debug build (compiled with -DDNS_CHECK, libdns_check.so):
// DNS_CK(status, cond, kernel, index) is true when cond holds; when it does not,
// the first failure of a launch is recorded in the group's device status word
// as BOUNDS_FLAG | kernel << 24 | (index & 0xFFFFFF) and the caller skips the
// access (no trap: the next synchronising call reports it).  Without
// DNS_CHECK the macro is the constant true and costs nothing.
constexpr int BOUNDS_FLAG = 0x40000000;
enum CheckKernel {
    CK_SELFTEST = 1, CK_SPEC = 2, CK_D2V = 3, CK_PLANE_LINES = 4, CK_YDERIV_T = 5, CK_FORCING_T = 6,
    CK_HELM_T = 7, CK_PACK = 8, CK_UNPACK = 9, CK_SPEC_SMEM = 10
};
__device__ __forceinline__ bool ck_record(int* status, bool ok, int kernel, long long index) {
    if (!ok) atomicCAS(status, 0, BOUNDS_FLAG | (kernel << 24) | (int)(index & 0xFFFFFF));
    return ok;
}
#ifdef DNS_CHECK
#define DNS_CK(status, cond, kernel, index) (::dnsk::ck_record((status), (cond), (kernel), (long long)(index)))
#else
#define DNS_CK(status, cond, kernel, index) (true)
#endif

template <typename T> struct C2;
template <> struct C2<double> { typedef double2 type; };
template <> struct C2<float> { typedef float2 type; };

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C, typename T>
__device__ __forceinline__ C cscale(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// i * a
template <typename C>
__device__ __forceinline__ C cmuli(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
template <typename C>
__device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

// Radix plan of one transform length N = 2^a 3^b <= 128.
struct FftPlan {
    int n;
    int nst;
    int rad[5];
};

// Radix-R DFT of v[0..R-1] in registers; SIGN = -1 forward, +1 inverse.
template <typename C, int SIGN>
__device__ __forceinline__ void butterfly(C* v, int R) {
    if (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b); v[1] = csub(a, b);
    } else if (R == 4) {
        C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        C c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        C id = cmuli(d);
        if (SIGN < 0) { id.x = -id.x; id.y = -id.y; }
        v[0] = cadd(a, c); v[2] = csub(a, c);
        v[1] = cadd(b, id); v[3] = csub(b, id);
    } else {  // R == 3
        typedef decltype(v[0].x) T;
        const T h = (T)0.86602540378443864676;   // sqrt(3)/2
        C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        C x0 = cadd(v[0], t1);
        C m; m.x = v[0].x - (T)0.5 * t1.x; m.y = v[0].y - (T)0.5 * t1.y;
        C s = cscale(cmuli(t2), (T)(SIGN) * h);
        v[0] = x0; v[1] = cadd(m, s); v[2] = csub(m, s);
    }
}

// CTA-wide Stockham FFT of nl lines of length p.n stored contiguously in b0
// (line stride p.n); b1 is scratch of the same size.  tw holds the forward
// twiddles exp(-2 pi i t / n), t < n.  Returns the buffer holding the result.
// Must be called by every thread of the CTA; ends with a __syncthreads.
template <typename C, int SIGN>
__device__ C* fft_lines(C* b0, C* b1, int nl, const FftPlan& p, const C* tw) {
    C* src = b0;
    C* dst = b1;
    const int N = p.n;
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.rad[s];
        const int nb = N / R;
        const int tstep = N / (Ns * R);
        for (int idx = threadIdx.x; idx < nl * nb; idx += blockDim.x) {
            int line = idx / nb;
            int j = idx - line * nb;
            const C* in = src + line * N;
            C* out = dst + line * N;
            int k = j % Ns;
            C v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < R) v[r] = in[j + r * nb];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < 4; ++r)
                    if (r < R) {
                        C w = tw[k * r * tstep];
                        if (SIGN > 0) w.y = -w.y;
                        v[r] = cmul(v[r], w);
                    }
            }
            butterfly<C, SIGN>(v, R);
            int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < R) out[base + r * Ns] = v[r];
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}

// Compile-time radix plan of length N, in the order make_plan builds it (a
// factor 3 first, then 4s, then a final 2): radix of stage s, number of stages.
__host__ __device__ constexpr int ct_radix(int N, int s) {
    int n = N, st = 0;
    if (n % 3 == 0) { if (st == s) return 3; ++st; n /= 3; }
    while (n % 4 == 0) { if (st == s) return 4; ++st; n /= 4; }
    if (n % 2 == 0) { if (st == s) return 2; ++st; n /= 2; }
    return 1;
}
__host__ __device__ constexpr int ct_stages(int N) {
    int s = 0;
    while (ct_radix(N, s) > 1) ++s;
    return s;
}

// fft_lines with the length, the line count and the plan known at compile
// time: the same stages and the same arithmetic in the same order (bitwise the
// same results), with the index divisions by constants.
template <typename C, int SIGN, int N, int NL, int S = 0, int NS = 1>
__device__ __forceinline__ C* fft_lines_ct(C* src, C* dst, const C* tw) {
    if constexpr (S == ct_stages(N)) {
        return src;
    } else {
        constexpr int R = ct_radix(N, S), NB = N / R, TSTEP = N / (NS * R);
        for (int idx = threadIdx.x; idx < NL * NB; idx += blockDim.x) {
            const int line = idx / NB, j = idx - line * NB;
            const C* in = src + line * N;
            C* out = dst + line * N;
            const int k = j % NS;
            C v[4];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = in[j + r * NB];
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[k * r * TSTEP];
                    if (SIGN > 0) w.y = -w.y;
                    v[r] = cmul(v[r], w);
                }
            }
            butterfly<C, SIGN>(v, R);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) out[base + r * NS] = v[r];
        }
        __syncthreads();
        return fft_lines_ct<C, SIGN, N, NL, S + 1, NS * R>(dst, src, tw);
    }
}

// Block-wide sum of a double (blockDim.x multiple of 32, <= 1024); result valid in
// every thread.  red must hold 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) {
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) red[0] = t;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) {
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (l == 0) red[0] = t;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// dU00/dy and dW00/dy at node row `row` (warp 0 of the CTA; result in out[0..1],
// valid after the caller's next __syncthreads).
__device__ __forceinline__ void mean_dy_row(const double* __restrict__ D1, const double* __restrict__ U,
                                            const double* __restrict__ W, int My, int row, double* out) {
    if (threadIdx.x >= 32) return;
    const double* d = D1 + (size_t)row * My;
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < My; j += 32) { a += d[j] * U[j]; b += d[j] * W[j]; }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

// Division by a divisor fixed for the whole kernel (Granlund and Montgomery,
// division by invariant integers): q = floor(n / d) = high 32 bits of n * M with
// M = floor((2^32 - 1) / d) + 1, exact whenever n * d < 2^32 (the error n * (M
// - 2^32 / d) / 2^32 then stays below 1/d).  One division per thread to set up,
// a multiply-high per use instead of the general integer division sequence.
struct FastDiv {
    unsigned d, M;
    __device__ __forceinline__ explicit FastDiv(unsigned dd) : d(dd), M(dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u) {}
    __device__ __forceinline__ unsigned div(unsigned n) const { return d > 1 ? __umulhi(n, M) : n; }
    __device__ __forceinline__ unsigned mod(unsigned n) const { return n - div(n) * d; }
};

// Allow a kernel the largest dynamic shared memory the SM offers next to its
// static shared memory (227 KB per block on sm_103).
template <typename F>
inline cudaError_t allow_max_dynamic_smem(F* func) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void*)func);
    if (e != cudaSuccess) return e;
    const int total = 227 * 1024;
    return cudaFuncSetAttribute((const void*)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                total - (int)a.sharedSizeBytes);
}

}  // namespace dnsk
