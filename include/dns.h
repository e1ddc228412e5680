/*
 * dns.h -- C ABI of the ensemble channel DNS step library (libdns.so).
 *
 * The library advances whole ensembles of plane Couette / plane Poiseuille
 * realisations by full Crank-Nicolson / 3rd-order Runge-Kutta time steps of the
 * wall-normal velocity / vorticity (v-eta) formulation, Fourier (x, z) x
 * Chebyshev (y) pseudo-spectral, on one CUDA GPU (sm_103a).
 *
 * Method (arXiv 2306.12739, "A vectorized Navier-Stokes ensemble direct
 * numerical simulation code for plane parallel flows"):
 *   - equations: Sec. 2, Eqs. (Dv), (eta), (U00), (W00) and the boundary
 *     conditions v = dv/dy = eta = 0, U00(+-1) = +-U_w, W00(+-1) = 0;
 *   - time scheme: Sec. 3.1 (three CN sub-steps of lengths h = 1/2, 1, 1 with
 *     the nonlinear terms combined as F0, 2F1 - F0, (F0 + 4F1 + F2)/6, always
 *     restarting from the state at t);
 *   - implicit solves as precomputed matrices: Sec. 3.2, Eqs. CN1-CN4;
 *   - 2/3-rule dealiasing and the u, w recovery from v, eta: Sec. 3.2.
 *
 * Conventions shared by every call
 *   * Grid of a group: Mx x My x Mz collocation points; y_j = -cos(pi j/(My-1)),
 *     j = 0..My-1 (ascending, walls at j = 0 and My-1); x_i = i Lx/Mx,
 *     z_k = k Lz/Mz.  Retained modes: n = 0..Kx, m = -Kz..Kz with
 *     Kx = (Mx-1)/3, Kz = (Mz-1)/3 (integer division), kx = n 2pi/Lx,
 *     kz = m 2pi/Lz.  Supported Mx, Mz: 16, 32, 48, 64, 128 (128 with 64 or 128
 *     only); 5 <= My <= 129.
 *   * Host state layout (dns_set_state / dns_get_state):
 *       v_hat, eta_hat : double complex, interleaved (re, im),
 *                        [member][My-2 interior y][2 Kz + 1 (m + Kz)][Kx + 1 (n)]
 *       U00, W00       : double [member][My] (all nodes, walls included)
 *     The (n, m) = (0, 0) entries of v_hat and eta_hat are ignored (zero).
 *   * Every call returns a dns_status (0 = success).  Nothing crosses the ABI as
 *     an exception.  dns_last_error() gives a one-line reason for the last
 *     failure on a handle.
 *   * Ownership: the handle owns its host copies of the operators.  ALL device
 *     memory is caller-owned: dns_workspace_size() says how much, the caller
 *     allocates it (e.g. a torch uint8 tensor) and binds it with
 *     dns_bind_workspace().  The CUDA stream is caller-owned too; every device
 *     operation of a handle is enqueued on that stream.
 *   * Asynchrony: dns_step() only enqueues work.  dns_get_state() and
 *     dns_stats() synchronise the stream before they return host data.
 */
#ifndef DNS_H
#define DNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DNS_OK = 0,
    DNS_ERR_INVALID = -1,     /* bad argument, bad configuration, unbound workspace */
    DNS_ERR_CUDA = -2,        /* a CUDA runtime call failed (message in dns_last_error) */
    DNS_ERR_NOMEM = -3,       /* workspace too small, host allocation failed */
    DNS_ERR_TIMEOUT = -4,     /* a bounded device wait gave up (reported by the next synchronising call) */
    DNS_ERR_NONFINITE = -5,   /* returned by dns_stats when any member holds NaN/Inf */
    DNS_ERR_UNSUPPORTED = -6  /* valid request the library does not implement */
} dns_status;

typedef enum { DNS_COUETTE = 0, DNS_POISEUILLE = 1 } dns_flow;

/* DNS_PREC_FP64: every stage in double precision (the comparator).
 * DNS_PREC_MIXED: transforms and nonlinear products in single precision, the
 * y-contractions and implicit applies in split precision, the boundary/mean-flow
 * solves and the state accumulation in double precision. */
typedef enum { DNS_PREC_FP64 = 0, DNS_PREC_MIXED = 1 } dns_precision;

/* One group: members that share grid, box, Re and dt. */
typedef struct {
    dns_flow flow;
    int mx, my, mz;        /* collocation points (x, y incl. both walls, z) */
    double lx, lz;         /* box lengths; Ly = 2 is fixed */
    double re;             /* Couette: half-gap wall speed; Poiseuille: laminar centreline speed */
    double dt;             /* fixed time step (the paper's scheme has no adaptive dt) */
    double u_wall;         /* Couette wall speed: U00(+-1) = +-u_wall (ignored for Poiseuille) */
    double bulk_flux;      /* Poiseuille: prescribed int_{-1}^{1} U00 dy (4/3 for U = 1 - y^2) */
    int members;           /* ensemble size of this group, >= 1 */
    int shared_mean;       /* 0: independent members.  1: the members share their
                              streamwise-mean (kx = 0) flow, an S3T-type ensemble (Sec. 4.1):
                              every sub-step the kx = 0 part of the nonlinear term and the
                              plane means <uv>, <wv> are replaced by their average over the
                              members, so the shared flow is driven by the ensemble-averaged
                              perturbation Reynolds stresses.  The caller sets the same kx = 0
                              part (n = 0 column of v, eta and U00, W00) for every member; it
                              then stays identical. */
    int nonlinear_form;    /* 0: advective N = u . grad u (Sec. 3.1).  1: rotational
                              N = omega x u; the v, eta forcings differ from the advective
                              ones only through the aliasing of the y collocation derivative
                              (the curl of grad |u|^2/2 vanishes), the mean flow is forced by
                              d/dy <uv>, <wv> in both.  Rotational needs fewer transforms
                              (6 inverse + 3 forward per plane); it is available for
                              Mx, Mz <= 64 (DNS_ERR_UNSUPPORTED otherwise). */
    int member_block;      /* independent members (shared_mean = 0) run internally as member
                              blocks of about this many members, each an independent branch
                              of the step that runs concurrently with the others on the GPU,
                              so that one block's last partial wave of CTAs overlaps another
                              block's work.  0: automatic, E/4 clamped to [4, 16] (one block
                              below 8 members).  Values >= members give one block; < 0 is
                              DNS_ERR_INVALID.  Shared-mean groups are always one block. */
    int linear;            /* 0: a DNS group.  1: a linearised disturbance ensemble (paper,
                              "Diagnostic utilities that benefit from vectorization" and
                              "Growth functional and linearized adjoint equations"): every
                              member is one disturbance of the single streamwise wavenumber
                              kx = kx_index 2 pi / lx with every kept kz, advanced by the
                              forward equations d/dt u' = -[(B . grad) u' + (u' . grad) B]
                              - grad p' + lap u' / Re, or by the adjoint equations in reversed
                              time (dns_set_direction), about the group's frozen
                              streamwise-mean base flow B (dns_set_base_flow; zero until set),
                              with the DNS's CN/RK3 scheme and step dt.  The state has one kx
                              column (dns_state_shape reports n_kx = 1) and no mean profiles:
                              U00, W00 are ignored by dns_set_state (may be NULL) and read as
                              zero.  mx, flow, u_wall, bulk_flux and member_block are ignored
                              (always one block); shared_mean and nonlinear_form must be 0. */
    int kx_index;          /* linear groups: n >= 1 (DNS_ERR_INVALID otherwise) */
} dns_group_desc;

/* Member blocks are invisible to the caller: results (bit for bit, for a given
 * kernel choice) and the group / member numbering of every call are the same
 * as for one block. */
typedef struct {
    int n_groups;                  /* >= 1 */
    const dns_group_desc* groups;  /* n_groups entries, copied by dns_create */
    dns_precision precision;
    int use_graph;                 /* 1: capture one full step as a CUDA graph and replay it */
    int persistent;                /* reserved, must be 0 */
    unsigned long long barrier_timeout_ns;  /* reserved, 0 */
    const char* autotune_cache;    /* optional text file: autotuner decisions are read from it
                                      and appended to it ("ygemm|plane|helm Mx My Mz E choice" for
                                      kernel variants, "spec_ec|spec_cta|ytile Mx My Mz E value"
                                      for the tile shapes: members per CTA of the fused stage,
                                      CTAs per SM of its parity-block form, first column-tile cap
                                      of the register-tiled y-derivatives; the shapes never change
                                      a result); NULL = none */
    int ygemm;                     /* mixed path y-derivatives of the step-by-step stage
                                      (helm 1-3, 8): 0 autotuned at dns_bind_workspace, 1
                                      register-tiled FP32 with D2 v summed in float-float, 2
                                      tcgen05 tensor cores with split-BF16 operands and FP32
                                      accumulation (groups with My <= 66 and <= 64 members), 3
                                      the register-tiled kernel of 1 in parity blocks (D1 and
                                      D2 as their even and odd halves; the same float-float
                                      D2 v).  The FP32 accumulation of 2 loses about 1e-5 of
                                      |D2 v| to the cancellation in D2's rows at My = 65, over
                                      the 1e-6 budget of the mixed step, so DNS groups time it
                                      against 1 and 3 only up to My = 49 (linear groups at every
                                      size); 1 and 3 are timed against each other at every size */
    int plane;                     /* plane stage: 0 autotuned where several kernels exist (else
                                      the only one; FP64 defaults to 1), 1 one CTA per plane
                                      (sizes <= 64), 2 a thread-block cluster per plane (64x64
                                      single precision, and every size with a 128), 3 one CTA
                                      per plane with each 1-D transform owned by one group of
                                      threads (mixed precision, sizes <= 64); a request for a
                                      variant the group's size lacks is ignored */
    int helm;                      /* mixed path per-wavenumber stage: 0 autotuned at
                                      dns_bind_workspace (DNS groups: 1, 2 and 8, each timed with
                                      the y-derivatives and the forcing, against 4 to 7; linear
                                      groups: 1 against 2),
                                      1 register-tiled FP32 implicit apply (one CTA per
                                      wavenumber pair and field), 2 tcgen05 tensor cores with
                                      split-BF16 operands (groups with My <= 66 and <= 64 members;
                                      others use 1), 3 register-tiled FP32 in persistent CTAs that
                                      copy the next pair's operators while computing the current
                                      (only on request: its grid fills the GPU, which in a step
                                      starves concurrent member blocks), 4 the fused stage: one
                                      launch per sub-step does the forcing, RK3 combination,
                                      implicit apply, the y-derivatives of the new state and the
                                      mean flow (DNS groups whose operators fit in shared memory:
                                      My <= 99; linear groups use 1 or 2), 5 the fused stage
                                      with D2 v of the new state computed inside the same launch
                                      (the tensor-core digit product of the separate D2 v
                                      kernel, bit for bit the same result; groups with
                                      My <= 66, at most 4 members per CTA; others run 4), 6 the
                                      fused stage in parity blocks: every operator (centro-
                                      symmetric M - I and P, anti-centro-symmetric D1 on the
                                      symmetric grid) applied as its even and odd halves, half
                                      the operator bytes and multiply-adds (groups whose D2 v
                                      comes from the tensor-core kernel; others run 4), 7 the
                                      same with D2 v summed inside it in float-float (D2 in
                                      parity blocks; every size the fused stage takes), 8 the
                                      step-by-step stage of 1 with its forcing (D1) and implicit
                                      apply (M - I, P) in parity blocks (DNS groups; linear
                                      groups and tiles that do not fit run 1) */
} dns_config;

/* One-point statistics of one member (paper Sec. 4), computed from the current
 * state at time t:
 *   e_total    volume-averaged kinetic energy (1/(2V)) int |u|^2 dV, mean flow included
 *   e_pert     the same without the (0, 0) mode
 *   tau_bottom, tau_top   dU00/dy at y = -1 and y = +1
 *   bulk_flux  int_{-1}^{1} U00 dy (Clenshaw-Curtis)
 *   gamma      Poiseuille pressure gradient of the last sub-step (0 for Couette)
 *   max_div    max over interior nodes and modes of |i kx u + dv/dy + i kz w|
 *   nonfinite  1 if any value of this member's state is NaN or Inf
 *   cfl        CFL number: dt times the maximum over the interior collocation
 *              points (the Mx x Mz grid of every interior plane) of
 *              |u|/dx + |v|/dy_j + |w|/dz, mean flow included, dx = Lx/Mx,
 *              dz = Lz/Mz, dy_j the smaller gap from node j to a neighbour
 *              (the velocity synthesised in single precision: about 1e-6
 *              relative); 0 for a linear group (disturbances of arbitrary
 *              amplitude)                                                    */
typedef struct {
    double e_total, e_pert, tau_bottom, tau_top, bulk_flux, gamma, max_div;
    int nonfinite;
    int reserved;
    double cfl;
} dns_stats_t;

typedef struct dns_handle dns_handle;

/* Validate the configuration and build every operator on the host (Sec. 3.2,
 * Listings 1 and 3: Chebyshev D, the clamped fourth derivative, and per
 * wavenumber pair and sub-step length the CN matrices M = A^{-1} B and
 * P = -h dt A^{-1} for v (Eq. CN1 multiplied through by Delta) and eta (Eq. CN2),
 * plus the mean-flow operators of Eqs. CN3/CN4), in double-double precision,
 * rounded once to double.  No device memory is touched.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: DNS_ERR_INVALID (bad config, message in *out's last error when *out
 * is returned, else none), DNS_ERR_UNSUPPORTED (grid size), DNS_ERR_NOMEM. */
int dns_create(const dns_config* cfg, void* cuda_stream, dns_handle** out);

/* Bytes of device memory the handle needs (operators, state, work arrays). */
int dns_workspace_size(const dns_handle* h, size_t* bytes);

/* Bind caller-owned device memory (>= dns_workspace_size bytes, 256-byte
 * aligned) and upload the operators on the handle's stream.  The memory must
 * stay valid until dns_destroy or the next bind.  Errors: DNS_ERR_NOMEM (too
 * small), DNS_ERR_INVALID (misaligned / NULL), DNS_ERR_CUDA. */
int dns_bind_workspace(dns_handle* h, void* dev_ptr, size_t bytes);

/* Sizes of group `group`: n_kx = Kx + 1 (1 for a linear group), n_kz = 2 Kz + 1,
 * ny_int = My - 2, my = My. */
int dns_state_shape(const dns_handle* h, int group, int* n_kx, int* n_kz, int* ny_int, int* my);

/* Copy `count` members starting at `member0` of group `group` into the library
 * (layout in the header comment).  ptr_kind: 0 = host pointers (pageable or
 * pinned), 1 = device pointers.  The n = 0 column is replaced by its Hermitian
 * part in m, x(0,m) := (x(0,m) + conj x(0,-m))/2 (the only part a real field
 * carries), and the (0,0) entries are zeroed (DNS groups; a linear group's
 * single column is stored as given).  Host pointers are read before
 * the call returns.
 * Transfer path: device buffers, and page-locked host buffers mapped into the
 * device's address space (cudaHostAlloc / pinned tensors; both ends of each
 * buffer are checked with cudaPointerGetAttributes), are read by the packing
 * kernel itself when v_hat, eta_hat are 16-byte and U00, W00 8-byte aligned:
 * one pass over the CPU-GPU link, no staging copy.  Pageable or less aligned
 * buffers are first copied into a device staging buffer.  Device buffers must
 * hold the whole range (count members), as for a copy.
 * Errors: DNS_ERR_INVALID (range, NULL, ptr_kind), DNS_ERR_CUDA. */
int dns_set_state(dns_handle* h, int group, int member0, int count,
                  const double* v_hat, const double* eta_hat,
                  const double* U00, const double* W00, int ptr_kind);

/* Copy members out (same layout; the same transfer paths, the unpacking
 * kernel writing device or mapped page-locked host buffers itself).  Any of
 * the four destinations may be NULL (not wanted).  Synchronises the stream. */
int dns_get_state(const dns_handle* h, int group, int member0, int count,
                  double* v_hat, double* eta_hat, double* U00, double* W00, int ptr_kind);

/* One group's whole state (all members), layouts as for dns_set_state /
 * dns_get_state.  In dns_state_out any pointer may be NULL (not wanted); U00
 * and W00 are not read for a linear group. */
typedef struct {
    const double* v_hat;
    const double* eta_hat;
    const double* U00;
    const double* W00;
} dns_state_in;
typedef struct {
    double* v_hat;
    double* eta_hat;
    double* U00;
    double* W00;
} dns_state_out;

/* Upload, advance and download in one call (host-transfer scheduling, no
 * counterpart in the paper; the steps are those of dns_step, Sec. 3.1): every
 * group's state is replaced by in[group] (in == NULL: keep the current state),
 * nsteps CN/RK3 steps run, and
 * the result is written to out[group] (out == NULL: nothing is read back).
 * Same results, bit for bit, as dns_set_state for every group, dns_step and
 * dns_get_state for every group; the difference is scheduling.  One exception:
 * on a member block whose stage the autotuner set to the fused per-wavenumber
 * stage (helm 0 in the config, decided 4-7), a call of at most 2 steps on the
 * direct path (captured whole, or eager) runs the block's step-by-step stage in
 * parity blocks (helm 8 with the tuned ygemm), which needs no derivatives of the
 * uploaded state, where the group's measured whole-step time on that stage
 * exceeds the fused one's by less, over the call's steps, than those
 * derivatives cost (timed at dns_bind_workspace); its results equal that
 * stage's, within the mixed budget of the fused one, and the block's next fused
 * step first computes the derivatives of its current state.  When every
 * buffer takes the direct path (device memory, mapped page-locked host memory;
 * see dns_set_state) each member block uploads, steps and downloads on its own
 * stream, the uploads one after another, so the link transfers of one block
 * overlap the computation of the others; with use_graph and nsteps <= 16 the
 * whole call is one CUDA graph, kept for the next call with the same buffers
 * and nsteps.  Otherwise (staged buffers, longer runs) it runs the uploads, the
 * steps and the downloads in sequence.  ptr_kind as for dns_set_state.
 * Synchronises the stream; host buffers may be reused when it returns.
 * Errors: DNS_ERR_INVALID (not bound, nsteps < 0, NULL inputs, ptr_kind),
 * DNS_ERR_CUDA, and the device status codes of dns_get_state. */
int dns_advance(dns_handle* h, int nsteps, const dns_state_in* in, const dns_state_out* out, int ptr_kind);

/* Enqueue nsteps full CN/RK3 steps of every group on the handle's stream. */
int dns_step(dns_handle* h, int nsteps);

/* Statistics of every member of `group` at the current time (synchronises).
 * per_member: [members] (required); ensemble_mean: arithmetic mean over the
 * group's members, except max_div and cfl (the largest over the members) and
 * nonfinite (any member) (optional); profiles: optional host array
 * [members][6][My] holding U00, W00, <u'u'>, <v'v'>, <w'w'>, <u'v'> (plane
 * averages; the perturbation parts vanish on the walls).
 * Returns DNS_ERR_NONFINITE (after filling the outputs) when any member of the
 * group holds a NaN or Inf. */
int dns_stats(dns_handle* h, int group, dns_stats_t* per_member, dns_stats_t* ensemble_mean,
              double* profiles);

/* Free the handle (not the caller's device memory).  Synchronises the stream. */
int dns_destroy(dns_handle* h);

/* Reason of the last failure on this handle ("" if none).  Valid until the
 * next call on the handle. */
const char* dns_last_error(const dns_handle* h);

/* Kernel variants `group` uses, after the autotuner ran (i.e. after
 * dns_bind_workspace): ygemm 1 register-tiled FP32 / 2 tcgen05 y-contraction /
 * 3 register-tiled FP32 in parity blocks;
 * plane 1 one CTA per plane / 2 a thread-block cluster per plane / 3 line-owned
 * single CTA per plane; helm 1 register-tiled FP32 / 2 tcgen05 implicit apply /
 * 3 persistent register-tiled FP32 / 4 the fused per-wavenumber stage / 5 the
 * fused stage with D2 v inside it / 6 the fused stage in parity blocks / 7 the
 * same with its float-float D2 v / 8 the register-tiled FP32 stage with its
 * forcing and apply in parity blocks.  Any output may be NULL. */
int dns_kernel_choice(const dns_handle* h, int group, int* ygemm, int* plane, int* helm);

/* Number of kernel launches enqueued by the last dns_step call (all steps). */
int dns_last_launch_count(const dns_handle* h);

/* Kernel classes reported by dns_step_timed, in launch order within a sub-step. */
enum {
    DNS_K_MEAN_DERIV = 0,  /* reserved (no kernel of this class any more; always 0) */
    DNS_K_YDERIV = 1,      /* Dv, D2v, D eta (shared Chebyshev operators) */
    DNS_K_PLANE = 2,       /* transforms + advective products + plane means */
    DNS_K_FORCING = 3,     /* F, G and the RK3 combination */
    DNS_K_HELM = 4,        /* per-wavenumber implicit apply */
    DNS_K_MEAN = 5,        /* mean flow + constant-flux gamma */
    DNS_K_SPEC = 6,        /* fused per-wavenumber stage (helm = 4): forcing, RK3 combination,
                              implicit apply, y-derivatives of the new state, mean flow */
    DNS_K_D2V = 7,         /* D2 v of the new state on tensor cores (with the fused stage, My <= 66) */
    DNS_K_NCLASS = 8
};

/* Like dns_step (never through a graph), with a CUDA event pair recorded on
 * the handle's stream around every kernel launch; synchronises, then returns
 * the summed device time in ms (ms[DNS_K_NCLASS]) and the number of launches
 * (launches[DNS_K_NCLASS]) of each kernel class over the nsteps steps. */
int dns_step_timed(dns_handle* h, int nsteps, double* ms, int* launches);

/* Self-test of the device-side timeout path: launches one kernel that waits,
 * with its usual iteration limit, on a barrier nobody arrives at; the wait
 * gives up, latches the device status word, and the call returns
 * DNS_ERR_TIMEOUT (the context stays usable).  Synchronises. */
int dns_selftest_timeout(dns_handle* h);

/* Bounds-checked debug build.  libdns_check.so is the same library compiled with
 * -DDNS_CHECK: the hot-path kernels check their global (and the fused stage its
 * shared-memory) indices; the first failing index of a launch and the kernel are
 * recorded in the group's device status word, the access is skipped (no trap),
 * and the next synchronising call returns DNS_ERR_CUDA with
 * "bounds check failed: kernel K, index I (mod 2^24)" in dns_last_error.
 * dns_checked_build returns 1 in that build, 0 in libdns.so.
 * dns_selftest_bounds enqueues one check whose condition is false (it touches no
 * memory) and synchronises: DNS_ERR_CUDA in the checked build, DNS_OK otherwise. */
int dns_checked_build(void);
int dns_selftest_bounds(dns_handle* h);

/* Host run of the integer-operation binary64 <-> binary32 conversions the
 * mixed-precision kernels apply to the FP64 state (the same source code the
 * device compiles): f_out[i] = d_in[i] rounded to nearest even (magnitudes
 * below 2^-126 give a signed zero), d_out[i] = f_in[i] exactly (binary32
 * subnormals give a signed zero).  Host pointers, n >= 0 elements each; no
 * handle, no device access.  No counterpart in the paper: it exists so the
 * conversions can be checked without a GPU. */
int dns_convert_selftest(const double* d_in, float* f_out, const float* f_in, double* d_out, long long n);

/* Host copies of what dns_create built, for inspection and tests; no device
 * access, valid before a workspace is bound.
 * dns_export_grid: y [My], D1 [My*My], D2 [My*My], D4c [(My-2)^2] and the
 *   Clenshaw-Curtis weights ccw [My] (Sec. 2, Listing 1; any output may be NULL).
 * dns_export_operators: the CN operators of Eqs. CN1/CN2 for sub-step length
 *   h = 1/2 (h_index 0) or h = 1 (h_index 1) and wavenumber pair
 *   pair = |m| (Kx + 1) + n, each (My-2)^2 doubles row-major (Listing 3). */
int dns_export_grid(const dns_handle* h, int group, double* y, double* D1, double* D2,
                    double* D4c, double* ccw);
int dns_export_operators(const dns_handle* h, int group, int h_index, int pair,
                         double* Mv, double* Pv, double* Me, double* Pe);

/* Allocation-free statistics.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at the moment they want
 * statistics -- a host that has handed all device memory to its own pool, an
 * embedding runtime that forbids cudaMalloc/cudaFree inside its step callback,
 * or a monitoring hook that must not wait on the allocator's device-wide
 * synchronisation.  It computes the same per-member statistics as dns_stats for
 * the current state of `group` and allocates nothing: the per-plane partial
 * sums go to a fixed array inside the library (2^20 doubles, 8 MiB, resident on
 * every GPU that loads the library until the process exits), everything else
 * uses the handle's bound workspace.
 *   out_dev: DEVICE pointer, [members][8] doubles per member, in this order:
 *            e_total, e_pert, tau_bottom, tau_top, bulk_flux, gamma, max_div,
 *            nonfinite (1.0 or 0.0).  Caller-owned.
 * Enqueued on the handle's stream; returns without synchronising.
 * dns_bind_workspace does this call's set-up, on the device that is current
 * there: it looks up the array's device address and loads the module that holds
 * the array and the statistics kernels.  With lazy module loading (the CUDA
 * default since 12.2) those loads are what takes device memory for the array
 * and the code, so they happen at bind time, never inside this call.  Every
 * call shares the one array, so
 * calls that overlap on the GPU (other streams, other handles) race; each call
 * writes every partial it reads, so nothing needs clearing between calls.
 * Errors: DNS_ERR_INVALID (unbound workspace, NULL output, or a group with
 * more than 2^20 / 6 member-planes -- members * (My - 2) > 174762; the
 * limit applies per member block, see dns_config, so in practice only a
 * shared-mean group can reach it),
 * DNS_ERR_CUDA (address lookup or launch failed). */
int dns_stats_noalloc(dns_handle* h, int group, double* out_dev);

/* ---- Linearised disturbance groups (dns_group_desc.linear = 1).
 * dns_stats of a linear group reports in e_pert (and e_total) the energy of
 * each disturbance, E = (1/4) sum_kz sum_j w_j (|u|^2 + |v|^2 + |w|^2) over the
 * interior Chebyshev nodes (w_j Clenshaw-Curtis weights): the volume average of
 * |u|^2 / 2 of the complex single-harmonic field. */

/* Frozen base flow of linear group `group`: U, V, W, each [My][Mz] row-major
 * on the Chebyshev nodes y_j (ascending, walls included) times the uniform
 * z_k = k lz / Mz.  Each field is truncated to the kept kz (|m| <= Kz) before
 * use, so that its products with the disturbances are free of aliasing; d/dy
 * is taken by the collocation derivative, d/dz spectrally.  (V, W) should be
 * divergence-free and every field but U zero at the walls; the library does not
 * check.  ptr_kind: 0 host, 1 device.  Synchronises the stream.
 * Errors: DNS_ERR_INVALID (not a linear group, NULL, non-finite values, unbound
 * workspace), DNS_ERR_CUDA. */
int dns_set_base_flow(dns_handle* h, int group, const double* U, const double* V, const double* W, int ptr_kind);

/* Equations the following dns_step calls advance linear group `group` with
 * (group = -1: every linear group): adjoint = 0 the forward linearised
 * equations, otherwise the adjoint equations (in reversed time).  Enqueued on
 * the stream (a captured step graph serves both directions).
 * Errors: DNS_ERR_INVALID (not a linear group, unbound workspace). */
int dns_set_direction(dns_handle* h, int group, int adjoint);

/* Modified Gram-Schmidt of the members of linear group `group`, in member
 * order, in the energy inner product (the one dns_stats reports): member k is
 * normalised after the projections on members 0..k-1 are removed.  norms
 * (optional host array [members]) receives each member's energy norm sqrt(E)
 * just before its normalisation; with norms the call synchronises, without it
 * it is only enqueued.  Errors: DNS_ERR_INVALID, DNS_ERR_CUDA. */
int dns_orthonormalize(dns_handle* h, int group, double* norms);

/* One iteration of the forward-adjoint optimal-growth method (Luchini 2000, as
 * the paper's optimal-disturbance ensembles use it) on a handle whose groups
 * are all linear: nsteps forward steps, nsteps adjoint steps starting from the
 * forward result, Gram-Schmidt (dns_orthonormalize) of every group; the
 * members are left orthonormal, ready for the next iteration, and the
 * direction forward.  gains (optional host array, the members of group 0, then
 * group 1, ...) receives the norms, which converge to the energy gains G_k =
 * E(T) / E(0) of the leading optimal disturbances (T = nsteps dt) once the
 * members have unit energy.  With gains the call synchronises.
 * Errors: DNS_ERR_INVALID (a non-linear group, nsteps < 1), DNS_ERR_CUDA. */
int dns_optimal_sweep(dns_handle* h, int nsteps, double* gains);

/* ---- Stochastic forcing of a DNS group (the paper's S3T ensemble run:
 * realisations mixed from eigenvectors of the diffusion operator acting on a
 * (Delta v, eta) state, scaled to equal diffusion rate, at one streamwise
 * wavenumber).  Structures: for kx = kx_index 2 pi / lx and every kept kz, the
 * n_eig least-damped eigenfunctions of d/dt Delta v = Delta Delta v / Re
 * (v = Dv = 0 at the walls: the even and odd Stokes modes) and n_eig of
 * d/dt eta = Delta eta / Re (eta = 0: sine modes), sampled at the Chebyshev
 * nodes and scaled to unit energy (the dns_stats inner product of one complex
 * kx column), so each injects energy at the same rate.  Every step, every
 * member receives sum_j xi_j f_j eps / sqrt(dt) with independent complex
 * unit-variance normals xi_j, held over the step's three sub-steps; eps is set
 * so that the mean injection rate of e_pert (dns_stats, which counts the +-kx
 * pair of the real field) is `rate` per member.  Random numbers: SplitMix64 on
 * counters (Steele, Lea & Flood 2014), 53-bit uniforms, Box-Muller; stream
 * `seed`, counter from (step, member, kz, block, structure), the step counted
 * from this call (a member's noise does not depend on member blocks).
 * rate = 0 switches the forcing off.  Invalidates a captured step graph (the
 * next dns_step captures again).  Synchronises the stream.
 * Errors: DNS_ERR_INVALID (linear group, kx_index outside 1..Kx, n_eig outside
 * 1..min(16, (My - 2) / 2), rate < 0 or not finite, unbound workspace). */
int dns_set_stochastic_forcing(dns_handle* h, int group, int kx_index, int n_eig, double rate,
                               unsigned long long seed);

/* Host copy of the forcing structures of kz index m_index (0 .. 2 Kz):
 * structures [2][n_eig][My - 2] (v block, then eta block), decay [2][n_eig]
 * their eigenvalues (negative, least damped first).  Either may be NULL. */
int dns_export_forcing(const dns_handle* h, int group, int m_index, double* structures, double* decay);

#ifdef __cplusplus
}
#endif
#endif /* DNS_H */
