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
// address).  That address is looked up, and the module holding the array and
// the statistics kernels are loaded, when a handle's workspace is bound
// (dns_bind_workspace, with the handle's device current): with lazy module
// loading those loads are where the device memory of the array and of the
// code is taken, so they happen there and not inside dns_stats_noalloc.
#include "../../include/dns.h"
#include "dns_internal.hpp"

#include <mutex>

namespace dnsk {

// 6 partial sums per (member, interior plane): max members * (My - 2) = 174762
constexpr size_t NOALLOC_MAX_PARTIALS = (size_t)1 << 20;

static __device__ __align__(256) double g_stats_scratch[NOALLOC_MAX_PARTIALS];

namespace {

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

// Set-up for the current device, run when a workspace is bound: resolves the
// array's address (loading this file's module, whose static data is the
// array) and loads the statistics kernels, so that under lazy module loading
// (CUDA_MODULE_LOADING=LAZY, the default since CUDA 12.2) the first
// dns_stats_noalloc call has nothing left to load or allocate.
cudaError_t noalloc_prepare() {
    double* p = nullptr;
    cudaError_t e = noalloc_scratch(&p);
    if (e != cudaSuccess) return e;
    return load_stats_kernels();
}

// The statistics of dns_stats (the FP64 y-derivatives, the per-plane sums and
// the per-member reduction, the same kernels), with the per-plane sums in the
// fixed array and the packed values in the caller's out; no profiles, no CFL.
void launch_stats_noalloc(const GroupView& g, double* scratch, double* out, cudaStream_t st) {
    launch_stats_packed(g, scratch, out, st);
}

}  // namespace dnsk
