// dns_stats_noalloc: the one-point statistics of dns_stats, enqueued without
// any allocation.  Some callers cannot allocate device memory when they need
// statistics: a host that has handed all device memory to its own pool or
// allocator up front, an embedding runtime that forbids cudaMalloc/cudaFree
// inside its per-step callback, or a monitoring hook that must not block on
// the allocator's device-wide synchronisation.  Here the per-plane partial
// sums, the only memory the reduction needs beyond the handle's bound
// workspace and the caller's output, live in a fixed array inside the library.
//
// The array: g_stats_scratch below, NOALLOC_MAX_PARTIALS doubles (8 MiB),
// resident on every GPU that loads the library until the process exits.
// Host code reaches it only through the address cudaGetSymbolAddress returns
// for the current device (the host-side name is a stand-in, not a device
// address); that address is looked up once per device, by the first call made
// on that device.
#include "../../include/dns.h"
#include "dns_internal.hpp"

#include <mutex>

namespace dnsk {

// 6 partial sums per (member, interior plane): max members * (My - 2) = 174762
constexpr size_t NOALLOC_MAX_PARTIALS = (size_t)1 << 20;

static __device__ __align__(256) double g_stats_scratch[NOALLOC_MAX_PARTIALS];

namespace {

// Per-plane Parseval sums of one (interior plane, member), written to part:
// uu, vv, ww, uv (perturbation, Sec. 4), max |div u|, non-finite flag.
__global__ void __launch_bounds__(256) k_na_plane(GroupView g, double* __restrict__ part) {
    __shared__ double red[32];
    const int y = blockIdx.x, e = blockIdx.y;
    const int Ny = g.ny, E = g.E, nmodes = g.nmodes, NKX = g.nkx;
    const size_t fs = (size_t)Ny * E * nmodes;
    const double2* P = g.P5d + ((size_t)y * E + e) * nmodes;
    double uu = 0, vv = 0, ww = 0, uv = 0, dmax = 0, nf = 0;
    const int q_mean = mean_mode(g);
    for (int q = threadIdx.x; q < nmodes; q += blockDim.x) {
        const double2 v = P[q], dv = P[fs + q], et = P[3 * fs + q];
        if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(et.x) || !isfinite(et.y)) nf = 1.0;
        if (q == q_mean) continue;
        const int mi = q / NKX, n = q - mi * NKX;
        const double kx = g.kxt[n], kz = g.kzt[mi], ki = g.k2inv[q];
        const double ax = (kx * dv.x - kz * et.x) * ki, ay = (kx * dv.y - kz * et.y) * ki;
        const double bx = (kz * dv.x + kx * et.x) * ki, by = (kz * dv.y + kx * et.y) * ki;
        const double2 u = make_double2(-ay, ax), w = make_double2(-by, bx);
        const double c = (n == 0 || g.lin) ? 1.0 : 2.0;   // real fields carry -kx too
        uu += c * (u.x * u.x + u.y * u.y);
        vv += c * (v.x * v.x + v.y * v.y);
        ww += c * (w.x * w.x + w.y * w.y);
        uv += c * (u.x * v.x + u.y * v.y);
        const double rx = -kx * u.y + dv.x - kz * w.y;
        const double ry = kx * u.x + dv.y + kz * w.x;
        dmax = fmax(dmax, sqrt(rx * rx + ry * ry));
    }
    uu = block_sum(uu, red); vv = block_sum(vv, red); ww = block_sum(ww, red);
    uv = block_sum(uv, red); dmax = block_max(dmax, red); nf = block_max(nf, red);
    if (threadIdx.x == 0) {
        double* o = part + ((size_t)e * Ny + y) * 6;
        o[0] = uu; o[1] = vv; o[2] = ww; o[3] = uv; o[4] = dmax; o[5] = nf;
    }
}

// Per-member reduction over y (Clenshaw-Curtis), packed as 8 doubles:
// e_total, e_pert, tau_bottom, tau_top, bulk_flux, gamma, max_div, nonfinite.
__global__ void k_na_final(GroupView g, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double red[32];
    const int e = blockIdx.x, Ny = g.ny, My = g.my;
    const double* U = g.U_t + (size_t)e * My;
    const double* W = g.W_t + (size_t)e * My;
    double ep = 0, em = 0, fl = 0, dm = 0, nf = 0;
    for (int j = threadIdx.x; j < My; j += blockDim.x) {
        double uu = 0, vv = 0, ww = 0;
        if (j > 0 && j < My - 1) {
            const double* s = part + ((size_t)e * Ny + (j - 1)) * 6;
            uu = s[0]; vv = s[1]; ww = s[2];
            dm = fmax(dm, s[4]);
            nf = fmax(nf, s[5]);
        }
        if (!isfinite(U[j]) || !isfinite(W[j])) nf = 1.0;
        const double w = g.ccw[j];
        ep += w * (uu + vv + ww);
        em += w * (U[j] * U[j] + W[j] * W[j]);
        fl += w * U[j];
    }
    ep = block_sum(ep, red); em = block_sum(em, red); fl = block_sum(fl, red);
    dm = block_max(dm, red); nf = block_max(nf, red);
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0;
        for (int j = 0; j < My; ++j) {
            t0 += g.D1[j] * U[j];
            t1 += g.D1[(size_t)(My - 1) * My + j] * U[j];
        }
        double* o = out + (size_t)e * 8;
        o[0] = 0.25 * (ep + em);
        o[1] = 0.25 * ep;
        o[2] = t0;
        o[3] = t1;
        o[4] = fl;
        o[5] = g.gamma[e];
        o[6] = dm;
        o[7] = nf;
    }
}

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};

}  // namespace

// Device address of the scratch array on the current device (looked up on the
// first call per device).  Returns cudaSuccess or the lookup's error.
cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stats_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

size_t noalloc_max_partials() { return NOALLOC_MAX_PARTIALS; }

void launch_stats_noalloc(const GroupView& g, double* scratch, double* out, cudaStream_t st) {
    launch_yderiv<double>(g, g.v_t, g.e_t, g.P5d, st);
    k_na_plane<<<dim3(g.ny, g.E), 256, 0, st>>>(g, scratch);
    k_na_final<<<g.E, 128, 0, st>>>(g, scratch, out);
}

}  // namespace dnsk
