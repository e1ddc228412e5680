// Stochastic forcing of a DNS group (the paper's S3T ensemble run, Sec.
// "Ensemble integrations": forcing realisations mixed from eigenvectors of the
// diffusion operator acting on a (Delta v, eta) state, scaled to equal
// diffusion rate, at one streamwise wavenumber).
//
// Once per step (before the forcing assembly of the first sub-step) this
// kernel draws, for every member, kz and structure, one complex unit-variance
// normal xi and forms the right-hand-side terms of the forced column
//   F_noise(y) = s sum_j xi_{v,j} (-Delta f_{v,j})(y),
//   G_noise(y) = s sum_j xi_{eta,j} (-f_{eta,j})(y),     s = eps / sqrt(dt),
// which the forcing kernels add in all three sub-steps (their combination
// weights sum to one, so a step receives the forcing once).  The structures
// are prepared on the host (dns_set_stochastic_forcing).
//
// Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) on counters -- draw k of seed
// s is mix64(s * 0xD1342543DE82EF95 + (k + 1) * 0x9E3779B97F4A7C15) -- as
// 53-bit uniforms on (0, 1), Box-Muller (cosine branch) from draws 2c, 2c + 1
// for the normal N(c); xi = (N(c) + i N(c + 1)) / sqrt(2),
// c = 2 (((((step E_group + member) NKZ + m) 2 + block) n_eig + j), with the
// member's index in its (user) group, so member blocks draw what one block would.
#include "dns_internal.hpp"

namespace dnsk {

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double sm64_uniform(unsigned long long seed, unsigned long long k) {
    const unsigned long long z = sm64_mix(seed * 0xD1342543DE82EF95ULL + (k + 1ULL) * 0x9E3779B97F4A7C15ULL);
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double sm64_normal(unsigned long long seed, unsigned long long c) {
    const double u1 = sm64_uniform(seed, 2ULL * c), u2 = sm64_uniform(seed, 2ULL * c + 1ULL);
    return sqrt(-2.0 * log(u1)) * cos((2.0 * 3.141592653589793) * u2);
}

// grid (NKZ, E), one CTA per (kz, member); 2 n_eig normals pairs in shared memory
__global__ void __launch_bounds__(128) k_stoch_noise(GroupView g) {
    __shared__ double2 xi[2 * STOCH_NEIG_MAX];
    const int mi = blockIdx.x, e = blockIdx.y;
    const int NKZ = g.nkz, J = g.fneig, Ny = g.ny, E = g.E;
    const unsigned long long step = *g.fstep;
    const unsigned long long member = (unsigned long long)(g.m0 + e);
    const double r2 = sqrt(2.0);
    for (int t = threadIdx.x; t < 2 * J; t += blockDim.x) {
        const int b = t / J, j = t - b * J;
        const unsigned long long idx =
            (((step * (unsigned long long)g.Eu + member) * NKZ + mi) * 2ULL + b) * (unsigned long long)J + j;
        const unsigned long long c = 2ULL * idx;
        xi[t] = make_double2(sm64_normal(g.fseed, c) / r2, sm64_normal(g.fseed, c + 1ULL) / r2);
    }
    __syncthreads();
    const double s = g.fscale;
    const double* bF = g.fbasis + (size_t)mi * 2 * J * Ny;
    const double* bG = bF + (size_t)J * Ny;
    const size_t half = (size_t)NKZ * Ny * E;
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) {
        double fx = 0.0, fy = 0.0, gx = 0.0, gy = 0.0;
        for (int j = 0; j < J; ++j) {
            const double a = bF[(size_t)j * Ny + y], b = bG[(size_t)j * Ny + y];
            fx += xi[j].x * a;
            fy += xi[j].y * a;
            gx += xi[J + j].x * b;
            gy += xi[J + j].y * b;
        }
        const size_t o = ((size_t)mi * Ny + y) * E + e;
        g.noise[o] = make_double2(s * fx, s * fy);
        g.noise[half + o] = make_double2(s * gx, s * gy);
    }
}

void launch_stoch_noise(const GroupView& g, cudaStream_t st) {
    k_stoch_noise<<<dim3(g.nkz, g.E), 128, 0, st>>>(g);
}

}  // namespace dnsk
