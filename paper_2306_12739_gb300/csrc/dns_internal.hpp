// Internal structures shared by the host orchestration and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "common.cuh"

namespace dnsk {

// Device-side view of one group.  Spectral arrays use two layouts:
//   H ("per-mode") layout  [q][y][e]  complex: the state, forcings and their
//                          accumulators; the block of mode q is a contiguous
//                          Ny x E complex matrix, i.e. the right-hand side of the
//                          per-wavenumber operators.
//   P ("per-plane") layout [y][e][q]  complex: inputs and outputs of the
//                          physical-space stage, one contiguous run of all modes
//                          per (plane, member).
// with q = (m + Kz) * NKX + n, NKX = Kx + 1, y the interior index 0..Ny-1.
struct GroupView {
    int mx, my, mz, kx, kz, nkx, nkz, nmodes, ny, E, npairs;
    int rp;               // Ny rounded up to a multiple of 4 (row padding of transposed operators)
    int kp;               // Ny rounded up to a multiple of 16 (K of the tensor-core y-contraction)
    int ygemm;            // mixed path y-derivatives: 1 register-tiled FP32, 2 tcgen05 split-BF16,
                          // 3 register-tiled FP32 in parity blocks; 0 = autotune
    int plane;            // plane stage: 1 single-CTA kernel, 2 cluster kernel, 3 line-owned
                          // single-CTA kernel (mixed path); 0 = autotune
    const void* Atc;      // tensor-core A image: [D1_int; D2_int] in 3 BF16 pieces
    int helm;             // mixed path implicit apply: 1 register-tiled FP32, 2 tcgen05, 3 persistent
                          // register-tiled FP32 with double-buffered operator copies, 4 the fused
                          // per-wavenumber stage (forcing, apply, y-derivatives, mean flow; 0 = autotune)
    const void* Htc[2];   // per h index: [npairs][2 fields] images of [M - I | P] in 3 BF16 pieces
    int* status;          // device error word (1: a bounded wait gave up)
    int flow;             // 0 Couette, 1 Poiseuille
    int shared_mean;      // 1: the members share the kx = 0 flow (forcing averaged over members)
    int rot;              // nonlinear term: 0 advective u . grad u, 1 rotational omega x u
    int lin;              // 1: linearised disturbance group: one kx != 0 column (nkx = 1, kxt[0]),
                          //    no mean mode, members are disturbance vectors
    int* dir;             // linear groups: device word, 0 forward equations, nonzero adjoint
    const double* base;   // linear groups: [9][Ny][Mz] U, V, W, d_y(U, V, W), d_z(U, V, W) of the
                          //    base flow on the interior planes
    const float* basef;   // single-precision copy (mixed path)
    double* gsr;          // linear groups: [E] energy norms recorded by the last Gram-Schmidt
    // stochastic forcing (DNS groups; fn = 0: off)
    int fn;               // forced streamwise index
    int fneig;            // structures per block (v, eta) and kz
    int m0, Eu;           // first member of this block in its group, members of the group
    int nblk;             // member blocks the group runs as (concurrent graph branches)
    double fscale;        // eps / sqrt(dt)
    unsigned long long fseed;
    const double* fbasis; // [NKZ][2][fneig][Ny] right-hand-side terms -Delta f_v, -f_eta
    double2* noise;       // [2][NKZ][Ny][E] this step's F and G terms of the forced column
    unsigned long long* fstep;   // device step counter of the noise
    double re, dt, u_wall, bulk_flux, lx, lz;
    FftPlan px, pz;
    // constants
    const double* D1;     // [My][My]
    const double* D1i;    // [Ny][Ny]
    const double* D2i;    // [Ny][Ny]
    const float* D1T;     // mixed path, transposed and row-padded: D1T[k][r] = D1i[r][k], [Ny][rp]
    const float* D2T;
    const float* D2Tl;    // D2T's residual: D2i - (double) D2T in single precision (compensated D2 v)
    int d2tc;             // fused stage: 1 = D2 v of the new state by the tensor-core digit kernel
    int d2fuse;           // fused stage: 1 = that digit product inside the fused launch (no D2 v launch)
    int spec_eo;          // fused stage: 1 = in parity blocks (even / odd parts in y; with d2tc)
    int spec_minb;        // fused stage in parity blocks: CTAs per SM of its register budget (2 or 3)
    int spec_eoff;        // fused stage in parity blocks: 1 = D2 v summed inside in float-float
    int step_eo;          // step-by-step stage (helm 1): 1 = forcing and implicit apply in parity blocks
    const float* opsEO[2];  // mixed path, per h index: [npairs][4] matrices (M - I, P of v and eta) in
                            // parity blocks, each eo_mat(Ny) floats (see k_spec.cu)
    const float* D1EO;      // D1 in parity blocks
    const float* D2EO;      // D2 in parity blocks and its residual D2 - (double) D2EO
    const float* D2lEO;
    int spec_ec;          // fused stage: members per CTA (0 = up to 8), set by the autotuner
    int yd_cap;           // register-tiled y-derivatives: first column-tile cap (0 = 64, or 32 above
                          //    Ny = 96), halved while the grid is short of 3 CTAs per SM; autotuned
    const void* D2oz;     // its image of D2: slices of 7-bit digits [64 rows][kp] (BF16)
    const int* D2ozexp;   // [64] row exponents of that image
    const double* ccw;    // [My]
    const double* kxt;    // [NKX]
    const double* kzt;    // [NKZ]
    const double* k2t;    // [nmodes]
    const double* k2inv;  // [nmodes], 0 at the mean mode
    const double2* twx;   // [Mx]
    const double2* twz;   // [Mz]
    const float2* twxf;
    const float2* twzf;
    const float* kxtf;
    const float* kztf;
    const float* k2invf;
    const double* ops[2];   // per h index: [npairs][4][Ny][Ny]  (Mv, Pv, Me, Pe)
    const float* opsfT[2];  // mixed path, per h index: [npairs][4][Ny][rp], transposed and row-padded
                            // single-precision (Mv - I), Pv, (Me - I), Pe
    const double* mops[2];  // per h index: MU [Ny][Ny], PU [Ny][Ny], bU [Ny][2], Ug [Ny], PD [Ny][My]
    // state, H layout
    double2 *v_t, *e_t, *v_s, *e_s;
    double2 *mx1_v, *mx1_e;       // M_1 x_t, shared by sub-steps 2 and 3
    double2 *Fv, *Fe, *Av, *Ae;   // combined forcing of this sub-step; RK accumulators
    double *U_t, *W_t, *U_s, *W_s;   // [E][My]
    double *AU, *AW;                 // RK accumulators of <uv>, <wv> [E][My]
    double *dU, *dW;                 // [E][My] scratch: pre-gamma mean profiles of the sub-step
    double *uv, *wv;                 // [E][My] plane means <uv>, <wv>
    double* gamma;                   // [E]
    int* mcnt;                       // [E] mean-flow row CTAs done in the current launch (fused stage)
    // P layout work arrays (element type by precision)
    void* P5;    // 5 fields: v, Dv, D2v, eta, Deta
    void* N3;    // 3 fields: Nu, Nv, Nw
    double2* P5d;  // FP64 copy for statistics (== P5 in FP64 mode)
    // statistics
    double* st_y;    // [E][Ny][6]: uu, vv, ww, uv, maxdiv, nonfinite
    double* st_out;  // [E][9] packed dns_stats_t doubles (+nonfinite as double, then the CFL number)
    double* cfl_y;   // [E][Ny] CFL rate (without dt) of every interior plane
    double* prof;    // [E][6][My]
    double2* stage;  // host-layout staging [E][Ny][nmodes] x 2 fields
};

// sprev >= 0: the launch also carries the mean-flow finish of sub-step sprev
template <typename T>
void launch_yderiv(const GroupView& g, const double2* v, const double2* e, void* P5, cudaStream_t st, int sprev = -1);
template <typename T>
void launch_plane_state(const GroupView& g, const double* U, const double* W, cudaStream_t st);
template <typename T>
void launch_forcing(const GroupView& g, int s, cudaStream_t st);
void launch_helm(const GroupView& g, int s, cudaStream_t st);
void launch_mean_finish(const GroupView& g, int s, cudaStream_t st);
// CTAs of the mean-flow rows carried by the implicit-apply launches (8 rows each)
__host__ __device__ inline int mean_row_ctas(const GroupView& g) { return g.lin ? 0 : g.E * ((g.ny + 7) / 8); }
// Members per CTA of the implicit-apply kernels (k_helm, k_helm_t).  A DNS
// group has hundreds of wavenumber pairs and keeps all its members in one CTA
// (operator reuse); a linear group has only Kz + 1 pairs, so its members are
// split into chunks until one group alone gives about one CTA per SM.
__host__ __device__ inline int helm_member_chunk(const GroupView& g) {
    if (!g.lin) return g.E;
    int want = (152 + 2 * g.npairs - 1) / (2 * g.npairs);
    if (want < 1) want = 1;
    if (want > g.E) want = g.E;
    return (g.E + want - 1) / want;
}
__host__ __device__ inline int helm_member_chunks(const GroupView& g) {
    const int ec = helm_member_chunk(g);
    return (g.E + ec - 1) / ec;
}
// index of the (0, 0) mode, or -1 in a linear group (which has none)
__host__ __device__ inline int mean_mode(const GroupView& g) { return g.lin ? -1 : g.kz * g.nkx; }
void launch_lin_plane(const GroupView& g, bool fp64, cudaStream_t st);
int launch_lin_orthonormalize(const GroupView& g, cudaStream_t st);   // returns the launch count
void set_attributes_linear();
constexpr int STOCH_NEIG_MAX = 16;   // forcing structures per block and kz
void launch_stoch_noise(const GroupView& g, cudaStream_t st);
inline size_t mean_smem_bytes(const GroupView& g) { return (8 * (size_t)g.my + 32) * sizeof(double); }
size_t helm_t_smem_bytes(const GroupView& g);
size_t yderiv_t_smem_bytes(const GroupView& g);
size_t forcing_t_smem_bytes(const GroupView& g);
void launch_yderiv_t(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev = -1);
void launch_forcing_t(const GroupView& g, int s, cudaStream_t st);
void launch_helm_t(const GroupView& g, int s, cudaStream_t st);
size_t helm_tp_smem_bytes(const GroupView& g);
void launch_helm_tp(const GroupView& g, int s, cudaStream_t st);
void set_attributes_gemm_t();
bool yderiv_tc_supported(const GroupView& g);
size_t yderiv_tc_smem_bytes(const GroupView& g);
void launch_yderiv_tc(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev = -1);
void set_attributes_yderiv_tc();
bool helm_tc_supported(const GroupView& g);
size_t helm_tc_smem_bytes(const GroupView& g);
void launch_helm_tc(const GroupView& g, int s, cudaStream_t st);
void set_attributes_helm_tc();
bool launch_plane_cl(const GroupView& g, bool fp64, const double* U, const double* W, cudaStream_t st);
size_t plane_cl_smem_bytes(int mx, int mz, bool fp64);
void set_attributes_plane_cl();
// D2 v on tensor cores with exact digit accumulation (k_d2v_tc.cu), Ny <= 64
bool d2v_tc_supported(const GroupView& g);
size_t d2v_tc_smem_bytes(const GroupView& g);
size_t d2v_tc_image_bytes(const GroupView& g);
void launch_d2v_tc(const GroupView& g, const double2* v, cudaStream_t st);
void set_attributes_d2v_tc();
// fused per-wavenumber stage of the mixed path (k_spec.cu)
bool spec_supported(const GroupView& g);
bool spec_d2fuse_supported(const GroupView& g);   // with g.d2fuse set: the fused D2 v can run
bool spec_eo_supported(const GroupView& g);       // the fused stage in parity blocks can run
size_t spec_eo_mat_floats(int ny);                // floats of one matrix in parity blocks
// the y-derivatives (and planes) of a newly set state for a group on the fused
// stage in parity blocks (D2 v with spec_eoff; else the digit kernel's)
void launch_eo_derivs(const GroupView& g, cudaStream_t st);
// one Ny x Ny row-major matrix (centro-symmetric, or anti-centro-symmetric when
// anti) as its two parity blocks, transposed and row-padded (out: spec_eo_mat_floats)
void spec_eo_image(const double* A, int ny, bool anti, float* out, bool residual = false);
size_t spec_smem_bytes(const GroupView& g);
void launch_spec(const GroupView& g, int s, cudaStream_t st);
void set_attributes_spec();
// the step-by-step y-derivatives, forcing and implicit apply in parity blocks (k_step_eo.cu)
bool yderiv_eo_supported(const GroupView& g);
size_t yderiv_eo_smem_bytes(const GroupView& g);
void launch_yderiv_eo(const GroupView& g, const double2* v, const double2* e, cudaStream_t st, int sprev = -1);
bool step_eo_supported(const GroupView& g);
size_t forcing_eo_smem_bytes(const GroupView& g);
size_t helm_eo_smem_bytes(const GroupView& g);
void launch_forcing_eo(const GroupView& g, int s, cudaStream_t st);
void launch_helm_eo(const GroupView& g, int s, cudaStream_t st);
void set_attributes_step_eo();
void launch_stats(const GroupView& g, cudaStream_t st);
// the statistics without profiles and CFL: per-plane sums into part [E][Ny][6],
// packed values into out [E][8]
void launch_stats_packed(const GroupView& g, double* part, double* out, cudaStream_t st);
cudaError_t load_stats_kernels();   // loads the kernels launch_stats_packed uses
void launch_shared_mean(const GroupView& g, bool fp64, cudaStream_t st);
void launch_pack(const GroupView& g, int member0, int count, const double2* sv, const double2* se, const double* sU,
                 const double* sW, cudaStream_t st);
void launch_unpack(const GroupView& g, int member0, int count, double2* dv, double2* de, double* dU, double* dW,
                   cudaStream_t st);
size_t plane_smem_bytes(const GroupView& g, int elem_bytes);
bool launch_plane_f32(const GroupView& g, const double* U, const double* W, cudaStream_t st);
size_t plane_f32_smem_bytes(int mx, int mz);
void set_attributes_plane_f32();
bool launch_plane_lines(const GroupView& g, const double* U, const double* W, cudaStream_t st);
size_t plane_lines_smem_bytes(int mx, int mz);
void set_attributes_plane_lines();
int plane_threads();

}  // namespace dnsk
