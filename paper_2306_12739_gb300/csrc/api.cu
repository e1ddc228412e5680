// C ABI of the ensemble channel DNS library: configuration, host-side operator
// build, workspace layout, state transfer and the CN/RK3 step orchestration
// (paper Sec. 3.1: three sub-steps, each = nonlinear evaluation, forcing
// combination, implicit per-wavenumber update, mean-flow update).
#include "../../include/dns.h"
#include "builder.hpp"
#include "dns_internal.hpp"
#include "cvt.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <cstdarg>
#include <string>
#include <thread>
#include <vector>

using dnsk::GroupView;

namespace {

// NVTX range over one library call (a named span on a profiler's host
// timeline; a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct HostGroup {
    dns_group_desc d;
    GroupView v;
    dnsb::GridOps grid;
    dnsb::CnOps ops[2];
    std::vector<double> kxt, kzt, k2t, k2inv, twx, twz, opsdev[2], mopsdev[2], D1i, D2i;
    std::vector<float> kxtf, kztf, k2invf, twxf, twzf, opsf[2], opsfT[2], D1T, D2T, D2Tl, opsEO[2], D1EO, D2EO, D2lEO;
    std::vector<uint16_t> Atc, Htc[2], D2oz;
    std::vector<int> D2ozexp;
    std::vector<double> fstruct, flam;   // stochastic forcing: structures [NKZ][2][n][Ny], decay rates
    // stochastic forcing: a side stream for the noise kernel, forked at the start
    // of every step and joined before the first forcing assembly
    cudaStream_t nstream = nullptr;
    cudaEvent_t nfork = nullptr, njoin = nullptr;
    cudaEvent_t uploaded = nullptr;   // this block's input is on the device (dns_advance)
    // dns_advance's short calls (at most ADVANCE_SBS_STEPS steps) on a block
    // whose autotuned stage is the fused one: the step-by-step stage in parity
    // blocks (vsbs: the same arrays, those variant flags), which needs no
    // derivatives of the uploaded state.  ygemm_sbs: the tuned y-derivative
    // variant the fused stage does not use.  p5_stale: such a call left the
    // per-plane arrays without the derivatives of the current state, which the
    // fused stage expects; the next fused step computes them first.
    GroupView vsbs{};
    bool has_sbs = false, p5_stale = false;
    int ygemm_sbs = 1;
    // whole-step times (ms per step of the handle) of the block's group on its
    // fused choice and on the step-by-step stage in parity blocks (0: unknown),
    // and the time of the derivatives of a newly set state of all its blocks
    float t_fused = 0.f, t_sbs = 0.f, t_derivs = 0.f;

    // byte offsets inside the workspace
    struct Off { size_t off, bytes; };
    std::vector<std::pair<void**, Off>> slots;
};

}  // namespace

struct dns_handle {
    dns_config cfg;
    std::vector<dns_group_desc> descs;
    std::string cache_path;
    std::vector<HostGroup> groups;     // internal groups (member blocks)
    // user group -> its member blocks: internal group index, first member, count
    struct Part { int ig, m0, E; };
    std::vector<std::vector<Part>> parts;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t need = 0;
    std::string err;
    int launches = 0;
    bool bound = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_launches = 0;
    // multi-group handles: one stream per group, forked from and joined back to
    // the caller's stream every step (independent branches of one graph)
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gevents;
    cudaEvent_t fork_ev = nullptr;
    // dns_advance as one graph, for the buffers and step count in akey
    cudaGraph_t agraph = nullptr;
    cudaGraphExec_t aexec = nullptr;
    std::vector<uintptr_t> akey;
    int alaunches = 0;
    int* hstatus = nullptr;   // page-locked copies of the groups' status words
};

// dns_advance calls of at most this many steps are captured whole
constexpr int ADVANCE_GRAPH_STEPS = 16;
// dns_advance calls of at most this many steps may run a fused-stage block on
// the step-by-step stage in parity blocks, where the group's measured step-time
// gap over the call's steps is below the derivatives of the uploaded state that
// the fused stage needs first (64x65x64 blocks of 4, one call per 0, 1, 2, 4
// steps: 171, 494, 844, 1538 us against 221, 545, 870, 1523 on the fused stage)
constexpr int ADVANCE_SBS_STEPS = 2;

namespace {

int fail(dns_handle* h, int code, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

bool make_plan(int N, dnsk::FftPlan* p) {
    p->n = N;
    p->nst = 0;
    int n = N;
    if (n % 3 == 0) { p->rad[p->nst++] = 3; n /= 3; }
    while (n % 4 == 0 && p->nst < 5) { p->rad[p->nst++] = 4; n /= 4; }
    if (n % 2 == 0 && p->nst < 5) { p->rad[p->nst++] = 2; n /= 2; }
    return n == 1;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool precision_mixed(const dns_handle* h) { return h->cfg.precision == DNS_PREC_MIXED; }

// the tcgen05 implicit apply may run: its operator images are needed
bool helm_tc_candidate(const GroupView& v) { return v.helm == 2 || (v.helm == 0 && dnsk::helm_tc_supported(v)); }
// the fused stage can run with its D2 v inside (helm request 5); v's own flag is untouched
bool d2fuse_ok(GroupView v) {
    v.d2fuse = 1;
    return dnsk::spec_d2fuse_supported(v);
}
// the fused stage can run in parity blocks, with D2 v from the digit kernel
// (helm request 6) or summed inside in float-float (ff, helm request 7)
bool eo_ok(GroupView v, bool ff) {
    v.spec_eo = 1;
    v.spec_eoff = ff ? 1 : 0;
    v.d2fuse = 0;
    return dnsk::spec_eo_supported(v);
}
// ... and its operator images are wanted (a request for it, or the autotuner)
bool eo_candidate(const GroupView& v) { return (v.helm == 4 || v.helm == 0) && eo_ok(v, true); }
// the step-by-step forcing and apply in parity blocks may run (a request, helm
// 8, or the autotuner): they read the pair operators and D1 in parity blocks
bool step_eo_candidate(const GroupView& v) {
    return (v.helm == 0 || (v.helm == 1 && v.step_eo)) && dnsk::step_eo_supported(v);
}
bool eo_images(const GroupView& v) { return eo_candidate(v) || step_eo_candidate(v); }

// Largest My at which DNS groups may take the FP32-accumulated tensor-core
// y-derivatives (see choose_variants)
constexpr int FP32_D2_MAX_MY = 49;

// the tcgen05 y-derivatives may run (a request, or the autotuner: DNS groups up
// to FP32_D2_MAX_MY, linear groups at every size): their operator image is needed
bool ygemm_tc_candidate(const GroupView& v) {
    return v.ygemm == 2 || (v.ygemm == 0 && dnsk::yderiv_tc_supported(v) && (v.lin || v.my <= FP32_D2_MAX_MY));
}
// the y-derivatives in parity blocks may run (a request, ygemm 3, or the
// autotuner): D1, D2 and its residual in parity blocks are needed
bool ygemm_eo_candidate(const GroupView& v) {
    return (v.ygemm == 0 || v.ygemm == 3) && dnsk::yderiv_eo_supported(v);
}

// Assign workspace offsets for every device array of group g (base = 0).
// The parity-block images of the fused stage in parity blocks: per h index and
// wavenumber pair, M_v - I, P_v, M_eta - I, P_eta (from the FP64 operators),
// and D1 (interior block).
// ops false: D1, D2 and its residual only (the y-derivatives in parity blocks).
void build_eo_images(HostGroup& G, bool ops) {
    const GroupView& v = G.v;
    const size_t nn = (size_t)v.ny * v.ny, mat = dnsk::spec_eo_mat_floats(v.ny);
    std::vector<double> a(nn);
    for (int hi = 0; hi < 2 && ops; ++hi) {
        G.opsEO[hi].assign((size_t)v.npairs * 4 * mat, 0.f);
        for (size_t blk = 0; blk < (size_t)v.npairs * 4; ++blk) {
            memcpy(a.data(), &G.opsdev[hi][blk * nn], nn * sizeof(double));
            if (blk % 4 == 0 || blk % 4 == 2)
                for (int i = 0; i < v.ny; ++i) a[(size_t)i * v.ny + i] -= 1.0;
            dnsk::spec_eo_image(a.data(), v.ny, false, &G.opsEO[hi][blk * mat]);
        }
    }
    G.D1EO.assign(mat, 0.f);
    dnsk::spec_eo_image(G.D1i.data(), v.ny, true, G.D1EO.data());
    G.D2EO.assign(mat, 0.f);
    G.D2lEO.assign(mat, 0.f);
    dnsk::spec_eo_image(G.D2i.data(), v.ny, false, G.D2EO.data());
    dnsk::spec_eo_image(G.D2i.data(), v.ny, false, G.D2lEO.data(), true);
}

size_t layout_group(dns_handle* h, HostGroup& G, size_t cur) {
    GroupView& v = G.v;
    G.slots.clear();
    auto add = [&](void** ptr, size_t bytes) {
        cur = align256(cur);
        G.slots.push_back({ptr, {cur, bytes}});
        cur += bytes;
    };
    const size_t S = (size_t)v.nmodes * v.ny * v.E;  // complex elements of one spectral field
    const size_t nn = (size_t)v.ny * v.ny;
    add((void**)&v.D1, sizeof(double) * v.my * v.my);
    add((void**)&v.D1i, sizeof(double) * nn);
    add((void**)&v.D2i, sizeof(double) * nn);
    add((void**)&v.D1T, sizeof(float) * (size_t)v.ny * v.rp);
    add((void**)&v.D2T, sizeof(float) * (size_t)v.ny * v.rp);
    add((void**)&v.D2Tl, sizeof(float) * (size_t)v.ny * v.rp);
    if (precision_mixed(h) && (eo_images(v) || ygemm_eo_candidate(v))) {
        add((void**)&v.D1EO, sizeof(float) * dnsk::spec_eo_mat_floats(v.ny));
        add((void**)&v.D2EO, sizeof(float) * dnsk::spec_eo_mat_floats(v.ny));
        add((void**)&v.D2lEO, sizeof(float) * dnsk::spec_eo_mat_floats(v.ny));
    }
    add((void**)&v.status, 256);
    if (ygemm_tc_candidate(v)) add((void**)&v.Atc, 3 * 128 * (size_t)v.kp * sizeof(uint16_t));
    if (v.d2tc) {
        add((void**)&v.D2oz, dnsk::d2v_tc_image_bytes(v));
        add((void**)&v.D2ozexp, 64 * sizeof(int));
    }
    add((void**)&v.ccw, sizeof(double) * v.my);
    add((void**)&v.kxt, sizeof(double) * v.nkx);
    add((void**)&v.kzt, sizeof(double) * v.nkz);
    add((void**)&v.k2t, sizeof(double) * v.nmodes);
    add((void**)&v.k2inv, sizeof(double) * v.nmodes);
    add((void**)&v.twx, sizeof(double2) * v.mx);
    add((void**)&v.twz, sizeof(double2) * v.mz);
    add((void**)&v.twxf, sizeof(float2) * v.mx);
    add((void**)&v.twzf, sizeof(float2) * v.mz);
    add((void**)&v.kxtf, sizeof(float) * v.nkx);
    add((void**)&v.kztf, sizeof(float) * v.nkz);
    add((void**)&v.k2invf, sizeof(float) * v.nmodes);
    for (int hi = 0; hi < 2; ++hi) {
        add((void**)&v.ops[hi], sizeof(double) * (size_t)v.npairs * 4 * nn);
        if (precision_mixed(h)) {
            add((void**)&v.opsfT[hi], sizeof(float) * (size_t)v.npairs * 4 * v.ny * v.rp);
            if (helm_tc_candidate(v)) add((void**)&v.Htc[hi], (size_t)v.npairs * 2 * 3 * 64 * 2 * v.kp * sizeof(uint16_t));
            if (eo_images(v)) add((void**)&v.opsEO[hi], sizeof(float) * (size_t)v.npairs * 4 * dnsk::spec_eo_mat_floats(v.ny));
        }
        add((void**)&v.mops[hi], sizeof(double) * (2 * nn + 3 * (size_t)v.ny + (size_t)v.ny * v.my));
    }
    double2** st[] = {&v.v_t, &v.e_t, &v.v_s, &v.e_s, &v.mx1_v, &v.mx1_e, &v.Fv, &v.Fe, &v.Av, &v.Ae};
    for (auto p : st) add((void**)p, sizeof(double2) * S);
    double** mf[] = {&v.U_t, &v.W_t, &v.U_s, &v.W_s, &v.dU, &v.dW, &v.uv, &v.wv};
    for (auto p : mf) add((void**)p, sizeof(double) * (size_t)v.E * v.my);
    add((void**)&v.AU, sizeof(double) * (size_t)v.E * v.my);
    add((void**)&v.AW, sizeof(double) * (size_t)v.E * v.my);
    add((void**)&v.gamma, sizeof(double) * v.E);
    add((void**)&v.mcnt, sizeof(int) * (size_t)v.E);
    if (!v.lin) {   // stochastic forcing (structures, one step's terms, the step counter)
        add((void**)&v.fbasis, sizeof(double) * (size_t)v.nkz * 2 * dnsk::STOCH_NEIG_MAX * v.ny);
        add((void**)&v.noise, sizeof(double2) * 2 * (size_t)v.nkz * v.ny * v.E);
        add((void**)&v.fstep, 256);
    }
    if (v.lin) {
        add((void**)&v.dir, 256);
        add((void**)&v.gsr, sizeof(double) * v.E);
        add((void**)&v.base, sizeof(double) * 9 * (size_t)v.ny * v.mz);
        if (precision_mixed(h)) add((void**)&v.basef, sizeof(float) * 9 * (size_t)v.ny * v.mz);
    }
    const size_t elem = precision_mixed(h) ? sizeof(float2) : sizeof(double2);
    add(&v.P5, elem * 5 * S);
    add(&v.N3, elem * 3 * S);
    if (precision_mixed(h)) add((void**)&v.P5d, sizeof(double2) * 5 * S);
    add((void**)&v.st_y, sizeof(double) * (size_t)v.E * v.ny * 6);
    add((void**)&v.st_out, sizeof(double) * (size_t)v.E * 9);
    add((void**)&v.cfl_y, sizeof(double) * (size_t)v.E * v.ny);
    add((void**)&v.prof, sizeof(double) * (size_t)v.E * 6 * v.my);
    add((void**)&v.stage, sizeof(double2) * 2 * S);
    return cur;
}

bool supported_m(int m) { return m == 16 || m == 32 || m == 48 || m == 64 || m == 128; }

int check(dns_handle* h, cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(h, DNS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return DNS_OK;
}

// A non-zero device status word as an error: a bounded wait that gave up
// (small codes), or, in the bounds-checked build, the first out-of-range index
// of a launch (dnsk::BOUNDS_FLAG | kernel << 24 | index & 0xFFFFFF).
int status_error(dns_handle* h, int sv) {
    if (sv & dnsk::BOUNDS_FLAG)
        return fail(h, DNS_ERR_CUDA, "bounds check failed: kernel %d, index %d (mod 2^24); the access was skipped",
                    (sv >> 24) & 0x3F, sv & 0xFFFFFF);
    return fail(h, DNS_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", sv);
}

// Read and clear the device status words after a synchronising call: a kernel
// whose bounded wait gave up latches 1 there.
int device_status(dns_handle* h) {
    for (auto& G : h->groups) {
        int st = 0;
        int rc = check(h, cudaMemcpy(&st, G.v.status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
        if (rc) return rc;
        if (st != 0) {
            cudaMemset(G.v.status, 0, sizeof(int));
            return status_error(h, st);
        }
    }
    return DNS_OK;
}

// The same check folded into a call's own synchronisation: the status words
// are copied into page-locked memory on stream st before it synchronises
// (one host round trip instead of one per member block), checked after.
int sync_with_status(dns_handle* h, cudaStream_t st, const char* what) {
    int rc;
    if (!h->hstatus &&
        (rc = check(h, cudaHostAlloc((void**)&h->hstatus, sizeof(int) * h->groups.size(), cudaHostAllocDefault),
                    "status buffer")))
        return rc;
    for (size_t ig = 0; ig < h->groups.size(); ++ig)
        if ((rc = check(h, cudaMemcpyAsync(h->hstatus + ig, h->groups[ig].v.status, sizeof(int), cudaMemcpyDeviceToHost,
                                           st), "read status")))
            return rc;
    if ((rc = check(h, cudaStreamSynchronize(st), what))) return rc;
    for (size_t ig = 0; ig < h->groups.size(); ++ig) {
        const int sv = h->hstatus[ig];
        if (sv != 0) {
            cudaMemset(h->groups[ig].v.status, 0, sizeof(int));
            return status_error(h, sv);
        }
    }
    return DNS_OK;
}

// Optional per-launch event recording (dns_step_timed).
struct Timer {
    std::vector<cudaEvent_t> ev;
    std::vector<int> cls;
};

void enqueue_group(dns_handle* h, HostGroup& G, cudaStream_t st, Timer* tm) {
    auto mark = [&](int c) {
        if (!tm) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        tm->ev.push_back(e);
        tm->cls.push_back(c);
    };
    const GroupView& g = G.v;
    // the step's noise depends only on the step counter: it is drawn beside the
    // y-derivatives and the plane stage (per-launch timing keeps it in line)
    const bool side_noise = g.fn > 0 && !tm && G.nstream;
    if (side_noise) {
        cudaEventRecord(G.nfork, st);
        cudaStreamWaitEvent(G.nstream, G.nfork, 0);
        dnsk::launch_stoch_noise(g, G.nstream);
        cudaEventRecord(G.njoin, G.nstream);
        h->launches += 1;
    }
    for (int s = 0; s < 3; ++s) {
        const double2* cv = s == 0 ? g.v_t : g.v_s;
        const double2* ce = s == 0 ? g.e_t : g.e_s;
        const double* cU = s == 0 ? g.U_t : g.U_s;
        const double* cW = s == 0 ? g.W_t : g.W_s;
        const int sprev = (s > 0 && !g.lin) ? s - 1 : -1;   // mean-flow finish carried by the y-derivatives
        mark(-1);
        if (precision_mixed(h) && g.helm == 4) {
            // the derivatives of this sub-step's state came with the previous
            // fused launch (or with the setting of the state)
            if (g.plane == 2) dnsk::launch_plane_cl(g, false, cU, cW, st);
            else if (g.plane == 3) dnsk::launch_plane_lines(g, cU, cW, st);
            else dnsk::launch_plane_f32(g, cU, cW, st);
            mark(DNS_K_PLANE);
            if (g.shared_mean && g.E > 1) { dnsk::launch_shared_mean(g, false, st); h->launches += 1; }
            if (s == 0 && g.fn > 0 && !side_noise) { dnsk::launch_stoch_noise(g, st); h->launches += 1; }
            if (s == 0 && side_noise) cudaStreamWaitEvent(st, G.njoin, 0);
            dnsk::launch_spec(g, s, st);
            mark(DNS_K_SPEC);
            h->launches += 2;
            if (g.d2tc && !g.d2fuse && !g.spec_eoff) {
                dnsk::launch_d2v_tc(g, s == 2 ? g.v_t : g.v_s, st);
                mark(DNS_K_D2V);
                h->launches += 1;
            }
            continue;
        }
        if (precision_mixed(h)) {
            if (g.ygemm == 2) dnsk::launch_yderiv_tc(g, cv, ce, st, sprev);
            else if (g.ygemm == 3) dnsk::launch_yderiv_eo(g, cv, ce, st, sprev);
            else dnsk::launch_yderiv_t(g, cv, ce, st, sprev);
            mark(DNS_K_YDERIV);
            if (g.lin) dnsk::launch_lin_plane(g, false, st);
            else if (g.plane == 2) dnsk::launch_plane_cl(g, false, cU, cW, st);
            else if (g.plane == 3) dnsk::launch_plane_lines(g, cU, cW, st);
            else dnsk::launch_plane_f32(g, cU, cW, st);
            mark(DNS_K_PLANE);
            if (g.shared_mean && g.E > 1) { dnsk::launch_shared_mean(g, false, st); h->launches += 1; }
            if (s == 0 && g.fn > 0 && !side_noise) { dnsk::launch_stoch_noise(g, st); h->launches += 1; }
            if (s == 0 && side_noise) cudaStreamWaitEvent(st, G.njoin, 0);
            if (g.helm == 1 && g.step_eo) dnsk::launch_forcing_eo(g, s, st);
            else dnsk::launch_forcing_t(g, s, st);
        } else {
            dnsk::launch_yderiv<double>(g, cv, ce, g.P5, st, sprev);
            mark(DNS_K_YDERIV);
            if (g.lin) dnsk::launch_lin_plane(g, true, st);
            else if (g.plane == 2) dnsk::launch_plane_cl(g, true, cU, cW, st);
            else dnsk::launch_plane_state<double>(g, cU, cW, st);
            mark(DNS_K_PLANE);
            if (g.shared_mean && g.E > 1) { dnsk::launch_shared_mean(g, true, st); h->launches += 1; }
            if (s == 0 && g.fn > 0 && !side_noise) { dnsk::launch_stoch_noise(g, st); h->launches += 1; }
            if (s == 0 && side_noise) cudaStreamWaitEvent(st, G.njoin, 0);
            dnsk::launch_forcing<double>(g, s, st);
        }
        mark(DNS_K_FORCING);
        // per-wavenumber implicit apply (and the rows of the mean-flow update)
        if (precision_mixed(h)) {
            if (g.helm == 2) dnsk::launch_helm_tc(g, s, st);
            else if (g.helm == 3) dnsk::launch_helm_tp(g, s, st);
            else if (g.step_eo) dnsk::launch_helm_eo(g, s, st);
            else dnsk::launch_helm_t(g, s, st);
        } else {
            dnsk::launch_helm(g, s, st);
        }
        mark(DNS_K_HELM);
        if (g.lin) {   // no mean flow
            h->launches += 4;
            continue;
        }
        // the mean-flow rows ran as leading CTAs of the implicit apply; gamma and
        // the profiles: the next sub-step's y-derivative launch carries them, the
        // last sub-step's (which completes the step's state) runs here
        if (s == 2) {
            dnsk::launch_mean_finish(g, s, st);
            mark(DNS_K_MEAN);
            h->launches += 1;
        }
        h->launches += 4;
    }
}

// One full step of every group.  With several groups (and no per-launch
// timing) each group runs on its own stream, forked from and joined back to
// the caller's stream, so the groups of an uneven batch proceed concurrently
// (and a captured graph holds one independent branch per group).
void enqueue_step(dns_handle* h, Timer* tm = nullptr) {
    if (tm || h->groups.size() == 1 || h->gstreams.empty()) {
        for (auto& G : h->groups) enqueue_group(h, G, h->stream, tm);
        return;
    }
    cudaEventRecord(h->fork_ev, h->stream);
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
        cudaStreamWaitEvent(h->gstreams[gi], h->fork_ev, 0);
        enqueue_group(h, h->groups[gi], h->gstreams[gi], nullptr);
        cudaEventRecord(h->gevents[gi], h->gstreams[gi]);
    }
    for (size_t gi = 0; gi < h->groups.size(); ++gi) cudaStreamWaitEvent(h->stream, h->gevents[gi], 0);
}

// ---- autotuner: per group, time the y-contraction variants on the bound
// workspace (the work is data independent) and keep the faster one.
std::string tune_key(const GroupView& v) {
    char b[128];
    snprintf(b, sizeof b, "ygemm %d %d %d %d", v.mx, v.my, v.mz, v.E);
    return b;
}

// plane-stage variants: 1 one CTA per plane, 2 a thread-block cluster per
// plane, 3 line-owned single CTA (single precision only)
bool plane_variant_ok(bool mixed, const GroupView& v, int c) {
    const size_t lim = 227 * 1024;
    // the rotational form exists in the line-owned kernel (single precision) and
    // the single-CTA FP64 kernel
    if (v.rot && !((mixed && c == 3) || (!mixed && c == 1))) return false;
    if (c == 1) {
        const size_t b = mixed ? dnsk::plane_f32_smem_bytes(v.mx, v.mz) : dnsk::plane_smem_bytes(v, 8);
        return (mixed ? b > 0 : (v.mx <= 64 && v.mz <= 64)) && b <= lim;
    }
    if (c == 2) {
        const size_t b = dnsk::plane_cl_smem_bytes(v.mx, v.mz, !mixed);
        return b > 0 && b <= lim;
    }
    if (c == 3) {
        const size_t b = mixed ? dnsk::plane_lines_smem_bytes(v.mx, v.mz) : 0;
        return b > 0 && b <= lim;
    }
    return false;
}

std::string tune_helm_key(const GroupView& v) {
    char b[128];
    snprintf(b, sizeof b, "helm %d %d %d %d", v.mx, v.my, v.mz, v.E);
    return b;
}

std::string tune_plane_key(const GroupView& v) {
    char b[128];
    snprintf(b, sizeof b, "plane %d %d %d %d", v.mx, v.my, v.mz, v.E);
    return b;
}

// the integer after key on its last line in the cache (0: none)
int cache_lookup_value(const char* path, const std::string& key) {
    if (!path) return 0;
    FILE* f = fopen(path, "r");
    if (!f) return 0;
    char line[256];
    int found = 0;
    while (fgets(line, sizeof line, f)) {
        std::string ln(line);
        if (ln.compare(0, key.size(), key) == 0 && ln.size() > key.size() + 1 && ln[key.size()] == ' ')
            found = atoi(ln.c_str() + key.size() + 1);
    }
    fclose(f);
    return found;
}

// a tile-shape decision: the chosen value and every candidate's time
void cache_store_shape(const char* path, const std::string& key, int choice, const std::vector<int>& vals,
                       const std::vector<float>& ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d   #", key.c_str(), choice);
    for (size_t i = 0; i < vals.size(); ++i) fprintf(f, " value %d %.4f ms", vals[i], ms[i]);
    fprintf(f, "\n");
    fclose(f);
}

int cache_lookup(const char* path, const std::string& key) {
    if (!path) return 0;
    FILE* f = fopen(path, "r");
    if (!f) return 0;
    char line[256];
    int found = 0;
    while (fgets(line, sizeof line, f)) {
        std::string ln(line);
        if (ln.compare(0, key.size(), key) == 0 && ln.size() > key.size() + 1 && ln[key.size()] == ' ') {
            int c = atoi(ln.c_str() + key.size() + 1);
            if (c >= 1 && c <= 8) found = c;
        }
    }
    fclose(f);
    return found;
}

// the time recorded for variant c on key's last line in the cache (0: none)
float cache_lookup_time(const char* path, const std::string& key, int c) {
    if (!path) return 0.f;
    FILE* f = fopen(path, "r");
    if (!f) return 0.f;
    char line[512];
    float found = 0.f;
    char tag[32];
    snprintf(tag, sizeof tag, "variant %d ", c);
    while (fgets(line, sizeof line, f)) {
        std::string ln(line);
        if (ln.compare(0, key.size(), key) != 0 || ln.size() <= key.size() + 1 || ln[key.size()] != ' ') continue;
        const size_t at = ln.find(tag);
        found = at == std::string::npos ? 0.f : (float)atof(ln.c_str() + at + strlen(tag));
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, int choice, const float* ms, int nvar) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d   #", key.c_str(), choice);
    for (int c = 1; c <= nvar; ++c) {
        if (ms[c] > 0.f) fprintf(f, " variant %d %.4f ms", c, ms[c]);
        else fprintf(f, " variant %d n/a", c);
    }
    fprintf(f, "\n");
    fclose(f);
}


// Kernel variants of one (internal) group from its sizes and the request in the
// config; 0 entries are decided by the autotuner at dns_bind_workspace.
int choose_variants(dns_handle* h, const dns_config* cfg, GroupView& v, int gi) {
    const dns_group_desc& d = h->descs[gi];
    // y-contraction variant: 1 register-tiled FP32, 2 tcgen05, 3 register-tiled
    // FP32 in parity blocks; 0 = decided by the autotuner when the workspace is
    // bound (where more than one candidate can run)
    // The tensor-core one accumulates D2 v in FP32, which loses about 1e-5 of
    // |D2 v| to the cancellation in D2's rows at My = 65 (max row sum of |D2_int|
    // 1.2e6; eta 2.2e-6 after 50 steps, over the 1e-6 budget) but not at My = 49
    // (3.8e5; 4.2e-7): DNS groups time it against the float-float register-tiled
    // kernel up to My = 49 and use the latter above; linear groups time both.
    v.ygemm = 1;
    if (precision_mixed(h)) {
        const bool tc = dnsk::yderiv_tc_supported(v), eo = dnsk::yderiv_eo_supported(v);
        if (cfg->ygemm == 2 && tc) v.ygemm = 2;
        else if (cfg->ygemm == 3 && eo) v.ygemm = 3;
        else if (cfg->ygemm == 0 && ((tc && (v.lin || v.my <= FP32_D2_MAX_MY)) || eo)) v.ygemm = 0;
    }
    // per-wavenumber stage: 1 register-tiled FP32 apply, 2 tcgen05, 3 persistent
    // register-tiled FP32 with double-buffered operator copies, 4 the fused
    // stage (5 to 7 its forms), 8 = 1 with the forcing and apply in parity
    // blocks; 0 = autotuned among 1, 2, 8 (each after the y-derivatives and the
    // forcing) and 4 to 7
    v.helm = 1;
    v.step_eo = 0;
    if (precision_mixed(h)) {
        if (cfg->helm >= 4 && cfg->helm <= 7) v.helm = dnsk::spec_supported(v) ? 4 : 0;
        else if (cfg->helm == 8) v.step_eo = dnsk::step_eo_supported(v) ? 1 : 0;   // 1 in parity blocks
        else if (cfg->helm == 0) v.helm = 0;
        else if (cfg->helm == 2 && dnsk::helm_tc_supported(v)) v.helm = 2;
        else if (cfg->helm == 3) v.helm = 3;
    }
    if (v.helm == 4) v.ygemm = 1;   // only the derivatives of a newly set state run separately
    // with the fused stage, D2 v of each new state on tensor cores where the rows fit
    v.d2tc = ((v.helm == 4 || v.helm == 0) && dnsk::spec_supported(v) && dnsk::d2v_tc_supported(v)) ? 1 : 0;
    // and, on request (helm 5) or by the autotuner, that digit product inside the fused launch
    v.d2fuse = (cfg->helm == 5 && v.helm == 4 && d2fuse_ok(v)) ? 1 : 0;
    // or the fused stage in parity blocks (helm 6)
    v.spec_eo = 0;
    v.spec_eoff = 0;
    if (v.helm == 4 && ((cfg->helm == 6 && v.d2tc && eo_ok(v, false)) || (cfg->helm == 7 && eo_ok(v, true)))) {
        v.spec_eo = 1;
        v.spec_eoff = cfg->helm == 7 ? 1 : 0;
    }
    v.spec_minb = 2;
    // plane-stage kernel: single CTA per plane where it fits, a thread-block
    // cluster (distributed shared memory) where it does not; where both exist
    // the autotuner decides at bind time
    const bool mixed = precision_mixed(h);
    if (v.lin) {
        v.plane = 4;   // the z-only linearised plane stage, the only one a linear group has
    } else {
        const bool ok[4] = {false, plane_variant_ok(mixed, v, 1), plane_variant_ok(mixed, v, 2),
                            plane_variant_ok(mixed, v, 3)};
        const int navail = ok[1] + ok[2] + ok[3];
        if (navail == 0)
            return fail(h, DNS_ERR_UNSUPPORTED, "group %d: no plane-stage kernel for %dx%d", gi, d.mx, d.mz);
        v.plane = navail == 1 ? (ok[1] ? 1 : ok[2] ? 2 : 3) : (mixed ? 0 : 1);
        if (navail > 1 && cfg->plane >= 1 && cfg->plane <= 3 && ok[cfg->plane]) v.plane = cfg->plane;
    }
    if (precision_mixed(h)) {
        size_t m1 = dnsk::helm_t_smem_bytes(v), m2 = dnsk::yderiv_t_smem_bytes(v), m3 = dnsk::forcing_t_smem_bytes(v);
        if (helm_tc_candidate(v) && dnsk::helm_tc_smem_bytes(v) > m1) m1 = dnsk::helm_tc_smem_bytes(v);
        if (v.helm == 3 && dnsk::helm_tp_smem_bytes(v) > m1) m1 = dnsk::helm_tp_smem_bytes(v);
        if (v.helm == 4 && dnsk::spec_smem_bytes(v) > m1) m1 = dnsk::spec_smem_bytes(v);
        if (v.d2tc && dnsk::d2v_tc_smem_bytes(v) > m1) m1 = dnsk::d2v_tc_smem_bytes(v);
        size_t mm = m1 > m2 ? m1 : m2;
        mm = mm > m3 ? mm : m3;
        if (mm > 227 * 1024)
            return fail(h, DNS_ERR_UNSUPPORTED, "group %d: spectral stage needs %zu B of shared memory", gi, mm);
    }
    return DNS_OK;
}

// number of member blocks a group runs as
// Number of member blocks of a group.  Several blocks run as concurrent graph
// branches: the dominant plane kernel launches planes x members CTAs, and at
// one or a few CTAs per SM its last wave is partly empty; a concurrent block
// fills it.  Blocks of E/4 members (4 to 16) measured best from 8 to 64 members.
int member_blocks(const dns_group_desc& d) {
    if (d.shared_mean || d.linear) return 1;
    int b = d.member_block;
    if (b <= 0) b = std::min(16, std::max(4, d.members / 4));
    return std::max(1, d.members / b);
}

}  // namespace

namespace dnsk {
std::vector<uint16_t> yderiv_tc_a_image(const std::vector<double>& D1i, const std::vector<double>& D2i, int ny, int kp);
std::vector<uint16_t> helm_tc_a_images(const std::vector<double>& ops, int npairs, int ny, int kp);
void launch_wait_selftest(int* status, cudaStream_t st);
void launch_bounds_selftest(int* status, cudaStream_t st);
void d2v_tc_image(const std::vector<double>& D2i, int ny, int kp, std::vector<uint16_t>& img, std::vector<int>& rexp);
cudaError_t noalloc_scratch(double** out);
size_t noalloc_max_partials();
cudaError_t noalloc_prepare();
void launch_stats_noalloc(const GroupView& g, double* scratch, double* out, cudaStream_t st);
void set_attributes_spectral();
void set_attributes_plane();
}

extern "C" {

int dns_create(const dns_config* cfg, void* cuda_stream, dns_handle** out) {
    if (!cfg || !out || cfg->n_groups < 1 || !cfg->groups) return DNS_ERR_INVALID;
    *out = nullptr;
    dns_handle* h = new (std::nothrow) dns_handle();
    if (!h) return DNS_ERR_NOMEM;
    h->cfg = *cfg;
    h->descs.assign(cfg->groups, cfg->groups + cfg->n_groups);
    h->cfg.groups = h->descs.data();
    if (cfg->autotune_cache) {
        h->cache_path = cfg->autotune_cache;
        h->cfg.autotune_cache = h->cache_path.c_str();
    }
    h->stream = (cudaStream_t)cuda_stream;
    *out = h;
    if (cfg->precision != DNS_PREC_FP64 && cfg->precision != DNS_PREC_MIXED)
        return fail(h, DNS_ERR_INVALID, "unknown precision %d", (int)cfg->precision);
    if (cfg->persistent != 0) return fail(h, DNS_ERR_UNSUPPORTED, "persistent launch not available");
    // Groups of 32 or more independent members run as member blocks of about 16
    // (internal groups, concurrent branches of the step graph); the API keeps
    // the caller's group and member numbering.
    h->parts.resize(cfg->n_groups);
    int nint = 0;
    for (int gi = 0; gi < cfg->n_groups; ++gi) nint += member_blocks(h->descs[gi]);
    h->groups.resize(nint);
    int nthreads = (int)std::thread::hardware_concurrency();
    if (nthreads < 1) nthreads = 1;
    size_t cur = 0;
    int ig = 0;
    for (int gi = 0; gi < cfg->n_groups; ++gi) {
        const int nb = member_blocks(h->descs[gi]);
        const int E = h->descs[gi].members, base = nb > 0 ? E / nb : 0, rem = nb > 0 ? E % nb : 0;
        const int ig0 = ig;
        int m0 = 0;
        for (int b = 0; b < nb; ++b, ++ig) {
        dns_group_desc d = h->descs[gi];
        d.members = base + (b < rem ? 1 : 0);
        h->parts[gi].push_back({ig, m0, d.members});
        m0 += d.members;
        HostGroup& G = h->groups[ig];
        if (b > 0) {
            // a further block of the same group: same grid and operators (and nblk)
            G = h->groups[ig0];
            G.d = d;
            G.v.E = d.members;
            int rcv = choose_variants(h, cfg, G.v, gi);
            if (rcv) return rcv;
            if (ygemm_tc_candidate(G.v) && G.Atc.empty()) G.Atc = dnsk::yderiv_tc_a_image(G.D1i, G.D2i, G.v.ny, G.v.kp);
            if (G.v.d2tc && G.D2oz.empty()) dnsk::d2v_tc_image(G.D2i, G.v.ny, G.v.kp, G.D2oz, G.D2ozexp);
            if (precision_mixed(h) && ((eo_images(G.v) && G.opsEO[0].empty()) ||
                                       (ygemm_eo_candidate(G.v) && G.D1EO.empty())))
                build_eo_images(G, eo_images(G.v));
            if (precision_mixed(h) && helm_tc_candidate(G.v) && G.Htc[0].empty())
                for (int hi = 0; hi < 2; ++hi)
                    G.Htc[hi] = dnsk::helm_tc_a_images(G.opsdev[hi], G.v.npairs, G.v.ny, G.v.kp);
            cur = layout_group(h, G, cur);
            continue;
        }
        G.d = d;
        if (d.linear != 0 && d.linear != 1) return fail(h, DNS_ERR_INVALID, "group %d: linear must be 0 or 1", gi);
        const bool lin = d.linear == 1;
        if (!lin && d.flow != DNS_COUETTE && d.flow != DNS_POISEUILLE)
            return fail(h, DNS_ERR_INVALID, "group %d: unknown flow", gi);
        if (!(d.re > 0) || !(d.dt > 0) || !(d.lx > 0) || !(d.lz > 0) || d.members < 1)
            return fail(h, DNS_ERR_INVALID, "group %d: re, dt, lx, lz must be > 0 and members >= 1", gi);
        if (lin && d.kx_index < 1) return fail(h, DNS_ERR_INVALID, "group %d: kx_index must be >= 1", gi);
        if (lin && (d.shared_mean != 0 || d.nonlinear_form != 0))
            return fail(h, DNS_ERR_INVALID, "group %d: a linear group has no shared mean or nonlinear form", gi);
        if (d.my < 5 || d.my > 129) return fail(h, DNS_ERR_UNSUPPORTED, "group %d: My=%d outside 5..129", gi, d.my);
        if ((!lin && !supported_m(d.mx)) || !supported_m(d.mz))
            return fail(h, DNS_ERR_UNSUPPORTED, "group %d: Mx, Mz must be 16, 32, 48, 64 or 128", gi);
        GroupView& v = G.v;
        memset(&v, 0, sizeof v);
        // a linear group has no x grid: one kx column, kxt[0] = kx_index * 2 pi / lx
        v.lin = lin ? 1 : 0;
        v.mx = lin ? 0 : d.mx; v.my = d.my; v.mz = d.mz;
        v.kx = lin ? 0 : (d.mx - 1) / 3; v.kz = (d.mz - 1) / 3;
        v.nkx = v.kx + 1; v.nkz = 2 * v.kz + 1;
        v.nmodes = v.nkx * v.nkz;
        v.ny = d.my - 2;
        v.E = d.members;
        v.nblk = nb;
        v.npairs = v.nkx * (v.kz + 1);
        v.rp = (v.ny + 3) / 4 * 4;
        v.kp = (v.ny + 15) / 16 * 16;
        v.flow = d.flow == DNS_POISEUILLE ? 1 : 0;
        if (d.shared_mean != 0 && d.shared_mean != 1)
            return fail(h, DNS_ERR_INVALID, "group %d: shared_mean must be 0 or 1", gi);
        v.shared_mean = d.shared_mean;
        if (d.nonlinear_form != 0 && d.nonlinear_form != 1)
            return fail(h, DNS_ERR_INVALID, "group %d: nonlinear_form must be 0 or 1", gi);
        if (d.member_block < 0) return fail(h, DNS_ERR_INVALID, "group %d: member_block must be >= 0", gi);
        v.rot = d.nonlinear_form;
        v.re = d.re; v.dt = d.dt; v.u_wall = d.u_wall; v.bulk_flux = d.bulk_flux;
        v.lx = d.lx; v.lz = d.lz;
        if ((!lin && !make_plan(d.mx, &v.px)) || !make_plan(d.mz, &v.pz))
            return fail(h, DNS_ERR_UNSUPPORTED, "group %d: no radix plan", gi);
        {
            int rcv = choose_variants(h, cfg, v, gi);
            if (rcv) return rcv;
        }
        // operators
        G.grid = dnsb::build_grid(d.my);
        double a1 = dnsb::fundamental(d.lx), a3 = dnsb::fundamental(d.lz);
        G.kxt.resize(v.nkx); G.kzt.resize(v.nkz);
        for (int n = 0; n < v.nkx; ++n) G.kxt[n] = (lin ? d.kx_index : n) * a1;
        for (int mi = 0; mi < v.nkz; ++mi) G.kzt[mi] = (mi - v.kz) * a3;
        G.k2t.resize(v.nmodes); G.k2inv.resize(v.nmodes);
        for (int mi = 0; mi < v.nkz; ++mi)
            for (int n = 0; n < v.nkx; ++n) {
                int q = mi * v.nkx + n;
                double kx = G.kxt[n], kz = G.kzt[mi];
                double k2 = kx * kx + kz * kz;
                G.k2t[q] = k2;
                G.k2inv[q] = k2 > 0 ? 1.0 / k2 : 0.0;
            }
        std::vector<double> pk2(v.npairs);
        for (int am = 0; am <= v.kz; ++am)
            for (int n = 0; n < v.nkx; ++n) {
                double kx = G.kxt[n], kz = am * a3;
                pk2[am * v.nkx + n] = kx * kx + kz * kz;
            }
        const double hs[2] = {0.5, 1.0};
        const size_t nn = (size_t)v.ny * v.ny;
        for (int hi = 0; hi < 2; ++hi) {
            if (!dnsb::build_cn(G.grid, pk2, d.dt, d.re, hs[hi], &G.ops[hi], nthreads))
                return fail(h, DNS_ERR_INVALID, "group %d: singular implicit operator", gi);
            auto& od = G.opsdev[hi];
            od.resize((size_t)v.npairs * 4 * nn);
            for (int p = 0; p < v.npairs; ++p) {
                memcpy(&od[((size_t)p * 4 + 0) * nn], &G.ops[hi].Mv[p * nn], nn * 8);
                memcpy(&od[((size_t)p * 4 + 1) * nn], &G.ops[hi].Pv[p * nn], nn * 8);
                memcpy(&od[((size_t)p * 4 + 2) * nn], &G.ops[hi].Me[p * nn], nn * 8);
                memcpy(&od[((size_t)p * 4 + 3) * nn], &G.ops[hi].Pe[p * nn], nn * 8);
            }
            if (precision_mixed(h)) {
                // single-precision copies for the increment form: M - I and P
                auto& of = G.opsf[hi];
                of.resize(od.size());
                for (int p = 0; p < v.npairs; ++p)
                    for (int k = 0; k < 4; ++k) {
                        const double* src = &od[((size_t)p * 4 + k) * nn];
                        float* dst = &of[((size_t)p * 4 + k) * nn];
                        for (size_t i = 0; i < nn; ++i) {
                            double val = src[i];
                            if ((k == 0 || k == 2) && (i % (v.ny + 1) == 0)) val -= 1.0;
                            dst[i] = (float)val;
                        }
                    }
                auto& ot = G.opsfT[hi];
                const size_t mt = (size_t)v.ny * v.rp;
                ot.assign((size_t)v.npairs * 4 * mt, 0.f);
                for (size_t blk = 0; blk < (size_t)v.npairs * 4; ++blk)
                    for (int r = 0; r < v.ny; ++r)
                        for (int k = 0; k < v.ny; ++k)
                            ot[blk * mt + (size_t)k * v.rp + r] = of[blk * nn + (size_t)r * v.ny + k];
                std::vector<float>().swap(of);
            }
            auto& md = G.mopsdev[hi];
            md.clear();
            md.insert(md.end(), G.ops[hi].MU.begin(), G.ops[hi].MU.end());
            md.insert(md.end(), G.ops[hi].PU.begin(), G.ops[hi].PU.end());
            md.insert(md.end(), G.ops[hi].bU.begin(), G.ops[hi].bU.end());
            md.insert(md.end(), G.ops[hi].Ug.begin(), G.ops[hi].Ug.end());
            md.insert(md.end(), G.ops[hi].PD.begin(), G.ops[hi].PD.end());
        }
        G.D1i.resize(nn); G.D2i.resize(nn);
        for (int i = 0; i < v.ny; ++i)
            for (int j = 0; j < v.ny; ++j) {
                G.D1i[(size_t)i * v.ny + j] = G.grid.D1[(size_t)(i + 1) * d.my + (j + 1)];
                G.D2i[(size_t)i * v.ny + j] = G.grid.D2[(size_t)(i + 1) * d.my + (j + 1)];
            }
        G.D1T.assign((size_t)v.ny * v.rp, 0.f);
        G.D2T.assign((size_t)v.ny * v.rp, 0.f);
        G.D2Tl.assign((size_t)v.ny * v.rp, 0.f);
        for (int r = 0; r < v.ny; ++r)
            for (int k = 0; k < v.ny; ++k) {
                const double d2 = G.D2i[(size_t)r * v.ny + k];
                G.D1T[(size_t)k * v.rp + r] = (float)G.D1i[(size_t)r * v.ny + k];
                G.D2T[(size_t)k * v.rp + r] = (float)d2;
                G.D2Tl[(size_t)k * v.rp + r] = (float)(d2 - (double)(float)d2);
            }
        if (ygemm_tc_candidate(v)) G.Atc = dnsk::yderiv_tc_a_image(G.D1i, G.D2i, v.ny, v.kp);
        if (v.d2tc) dnsk::d2v_tc_image(G.D2i, v.ny, v.kp, G.D2oz, G.D2ozexp);
        if (precision_mixed(h) && (eo_images(v) || ygemm_eo_candidate(v))) build_eo_images(G, eo_images(v));
        if (precision_mixed(h) && helm_tc_candidate(v))
            for (int hi = 0; hi < 2; ++hi) G.Htc[hi] = dnsk::helm_tc_a_images(G.opsdev[hi], v.npairs, v.ny, v.kp);
        if (!lin) G.twx = dnsb::twiddles(d.mx);
        G.twz = dnsb::twiddles(d.mz);
        G.twxf.assign(G.twx.begin(), G.twx.end());
        G.twzf.assign(G.twz.begin(), G.twz.end());
        G.kxtf.assign(G.kxt.begin(), G.kxt.end());
        G.kztf.assign(G.kzt.begin(), G.kzt.end());
        G.k2invf.assign(G.k2inv.begin(), G.k2inv.end());
        cur = layout_group(h, G, cur);
        }
    }
    h->need = align256(cur);
    return DNS_OK;
}

int dns_workspace_size(const dns_handle* h, size_t* bytes) {
    if (!h || !bytes) return DNS_ERR_INVALID;
    *bytes = h->need;
    return DNS_OK;
}

// Captured graphs hold the group views (workspace pointers, forcing set-up):
// every change of those drops them, and the next step captures anew.
static void drop_graphs(dns_handle* h) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    if (h->aexec) { cudaGraphExecDestroy(h->aexec); h->aexec = nullptr; }
    if (h->agraph) { cudaGraphDestroy(h->agraph); h->agraph = nullptr; }
    h->akey.clear();
}

static int new_state_derivatives(dns_handle* h, const GroupView& v, cudaStream_t st);

int dns_bind_workspace(dns_handle* h, void* dev_ptr, size_t bytes) {
    NvtxRange range_("dns_bind_workspace");
    if (!h) return DNS_ERR_INVALID;
    if (!dev_ptr || ((uintptr_t)dev_ptr & 255)) return fail(h, DNS_ERR_INVALID, "workspace NULL or not 256-byte aligned");
    if (bytes < h->need) return fail(h, DNS_ERR_NOMEM, "workspace has %zu bytes, needs %zu", bytes, h->need);
    h->ws = (char*)dev_ptr;
    h->ws_bytes = bytes;
    drop_graphs(h);
    if (h->groups.size() > 1 && h->gstreams.empty()) {
        int rc0 = check(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming), "fork event");
        if (rc0) return rc0;
        for (size_t gi = 0; gi < h->groups.size(); ++gi) {
            cudaStream_t s2;
            cudaEvent_t e2;
            if ((rc0 = check(h, cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "group stream"))) return rc0;
            if ((rc0 = check(h, cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "group event"))) return rc0;
            h->gstreams.push_back(s2);
            h->gevents.push_back(e2);
        }
    }
    dnsk::set_attributes_spectral();
    dnsk::set_attributes_plane();
    dnsk::set_attributes_plane_f32();
    dnsk::set_attributes_gemm_t();
    dnsk::set_attributes_yderiv_tc();
    dnsk::set_attributes_plane_cl();
    dnsk::set_attributes_plane_lines();
    dnsk::set_attributes_helm_tc();
    dnsk::set_attributes_linear();
    dnsk::set_attributes_spec();
    dnsk::set_attributes_step_eo();
    dnsk::set_attributes_d2v_tc();
    {
        int rc0 = check(h, cudaGetLastError(), "kernel attributes");
        if (rc0) return rc0;
        // the fixed array of dns_stats_noalloc and its kernels, resolved and loaded now
        if ((rc0 = check(h, dnsk::noalloc_prepare(), "dns_stats_noalloc set-up"))) return rc0;
    }
    cudaStream_t st = h->stream;
    int rc = check(h, cudaMemsetAsync(dev_ptr, 0, h->need, st), "clear workspace");
    if (rc) return rc;
    for (auto& G : h->groups) {
        for (auto& s : G.slots) *s.first = h->ws + s.second.off;
        GroupView& v = G.v;
        if (!precision_mixed(h)) v.P5d = (double2*)v.P5;
        struct Up { const void* dst; const void* src; size_t bytes; };
        const Up ups[] = {
            {v.D1, G.grid.D1.data(), G.grid.D1.size() * 8},
            {v.D1i, G.D1i.data(), G.D1i.size() * 8},
            {v.D2i, G.D2i.data(), G.D2i.size() * 8},
            {v.ccw, G.grid.ccw.data(), G.grid.ccw.size() * 8},
            {v.kxt, G.kxt.data(), G.kxt.size() * 8},
            {v.kzt, G.kzt.data(), G.kzt.size() * 8},
            {v.k2t, G.k2t.data(), G.k2t.size() * 8},
            {v.k2inv, G.k2inv.data(), G.k2inv.size() * 8},
            {v.twx, G.twx.data(), G.twx.size() * 8},
            {v.twz, G.twz.data(), G.twz.size() * 8},
            {v.twxf, G.twxf.data(), G.twxf.size() * 4},
            {v.twzf, G.twzf.data(), G.twzf.size() * 4},
            {v.kxtf, G.kxtf.data(), G.kxtf.size() * 4},
            {v.kztf, G.kztf.data(), G.kztf.size() * 4},
            {v.k2invf, G.k2invf.data(), G.k2invf.size() * 4},
            {v.ops[0], G.opsdev[0].data(), G.opsdev[0].size() * 8},
            {v.ops[1], G.opsdev[1].data(), G.opsdev[1].size() * 8},
            {v.opsfT[0], G.opsfT[0].data(), G.opsfT[0].size() * 4},
            {v.opsfT[1], G.opsfT[1].data(), G.opsfT[1].size() * 4},
            {v.D1T, G.D1T.data(), G.D1T.size() * 4},
            {v.Atc, G.Atc.data(), G.Atc.size() * 2},
            {v.Htc[0], G.Htc[0].data(), G.Htc[0].size() * 2},
            {v.Htc[1], G.Htc[1].data(), G.Htc[1].size() * 2},
            {v.D2T, G.D2T.data(), G.D2T.size() * 4},
            {v.D2Tl, G.D2Tl.data(), G.D2Tl.size() * 4},
            {v.D2oz, G.D2oz.data(), G.D2oz.size() * 2},
            {v.opsEO[0], G.opsEO[0].data(), G.opsEO[0].size() * 4},
            {v.opsEO[1], G.opsEO[1].data(), G.opsEO[1].size() * 4},
            {v.D1EO, G.D1EO.data(), G.D1EO.size() * 4},
            {v.D2EO, G.D2EO.data(), G.D2EO.size() * 4},
            {v.D2lEO, G.D2lEO.data(), G.D2lEO.size() * 4},
            {v.D2ozexp, G.D2ozexp.data(), G.D2ozexp.size() * 4},
            {v.mops[0], G.mopsdev[0].data(), G.mopsdev[0].size() * 8},
            {v.mops[1], G.mopsdev[1].data(), G.mopsdev[1].size() * 8},
        };
        for (const auto& u : ups) {
            if (u.bytes == 0 || u.dst == nullptr) continue;
            rc = check(h, cudaMemcpyAsync((void*)u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, st), "upload operators");
            if (rc) return rc;
        }
    }
    rc = check(h, cudaStreamSynchronize(st), "bind workspace");
    if (rc) return rc;
    // decisions of this call by key: the member blocks of a group (and equal
    // groups) are tuned once and share the choice
    std::map<std::string, int> decided;
    std::map<std::string, std::pair<float, float>> decided_t;   // per-stage key: (chosen, step-by-step in parity) ms
    for (auto& G : h->groups) {
        GroupView& v = G.v;
        if (v.plane != 0) continue;
        const std::string key = tune_plane_key(v);
        int choice = decided.count(key) ? decided[key] : cache_lookup(h->cfg.autotune_cache, key);
        if (choice && !plane_variant_ok(true, v, choice)) choice = 0;   // a cache entry this group cannot run
        if (!choice) {
            float best[4] = {0.f, 0.f, 0.f, 0.f};
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int cand = 1; cand <= 3; ++cand) {
                if (!plane_variant_ok(true, v, cand)) continue;
                auto run = [&]() {
                    if (cand == 2) dnsk::launch_plane_cl(v, false, v.U_t, v.W_t, st);
                    else if (cand == 3) dnsk::launch_plane_lines(v, v.U_t, v.W_t, st);
                    else dnsk::launch_plane_f32(v, v.U_t, v.W_t, st);
                };
                for (int w = 0; w < 2; ++w) run();
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5; ++r) run();
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune plane");
                if (rc) break;
                cudaEventElapsedTime(&best[cand], e0, e1);
                best[cand] /= 5.f;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            choice = 0;
            for (int cand = 1; cand <= 3; ++cand)
                if (best[cand] > 0.f && (choice == 0 || best[cand] < best[choice])) choice = cand;
            cache_store(h->cfg.autotune_cache, key, choice, best, 3);
        }
        decided[key] = choice;
        v.plane = choice;
    }
    for (auto& G : h->groups) {
        GroupView& v = G.v;
        if (v.ygemm != 0) continue;
        const std::string key = tune_key(v);
        int choice = decided.count(key) ? decided[key] : cache_lookup(h->cfg.autotune_cache, key);
        // candidates: 1 always; 2 where its operator image was laid out; 3 where
        // the parity-block images were
        const bool tc_ok = ygemm_tc_candidate(v) && v.Atc != nullptr;
        const bool eo_ok3 = ygemm_eo_candidate(v) && v.D1EO != nullptr && v.D2EO != nullptr && v.D2lEO != nullptr;
        if (choice > 3 || (choice == 2 && !tc_ok) || (choice == 3 && !eo_ok3)) choice = 0;
        if (!choice) {
            float best[4] = {0.f, 0.f, 0.f, 0.f};
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int cand = 1; cand <= 3; ++cand) {
                if ((cand == 2 && !tc_ok) || (cand == 3 && !eo_ok3)) continue;
                auto run = [&]() {
                    if (cand == 2) dnsk::launch_yderiv_tc(v, v.v_t, v.e_t, st);
                    else if (cand == 3) dnsk::launch_yderiv_eo(v, v.v_t, v.e_t, st);
                    else dnsk::launch_yderiv_t(v, v.v_t, v.e_t, st);
                };
                for (int w = 0; w < 2; ++w) run();
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5; ++r) run();
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune");
                if (rc) break;
                cudaEventElapsedTime(&best[cand], e0, e1);
                best[cand] /= 5.f;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            choice = 1;
            for (int cand = 2; cand <= 3; ++cand)
                if (best[cand] > 0.f && best[cand] < best[choice]) choice = cand;
            cache_store(h->cfg.autotune_cache, key, choice, best, 3);
        }
        decided[key] = choice;
        v.ygemm = choice;
    }
    // The per-wavenumber stage of a DNS group (step-by-step SIMT or tcgen05
    // apply, or the fused stage) is chosen by timing whole steps of the handle,
    // every member block of the group on the candidate: what it costs inside
    // the step graph, where member blocks and groups run concurrently, is not
    // what a kernel costs alone (the 64-member 32x49x32 Couette blocks: the
    // fused stage wins alone, the step-by-step stage by 20 % in the step).
    // Groups still undecided run the SIMT apply meanwhile.
    for (size_t gi = 0; gi < h->parts.size(); ++gi) {
        GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
        if (v0.lin || v0.helm != 0) continue;
        const std::string key = tune_helm_key(v0);
        int choice = decided.count(key) ? decided[key] : cache_lookup(h->cfg.autotune_cache, key);
        // 5: the fused stage with its D2 v inside (every block of the group must allow it)
        // 6, 7: the fused stage in parity blocks, D2 v by the digit kernel or
        // inside in float-float (its images were laid out for every block)
        // 8: the step-by-step stage with its forcing and apply in parity blocks
        bool fuse_ok = dnsk::spec_supported(v0), par_ok = dnsk::spec_supported(v0), ff_ok = par_ok, seo_ok = true;
        for (const auto& P : h->parts[gi]) {
            const GroupView& vb = h->groups[P.ig].v;
            fuse_ok = fuse_ok && d2fuse_ok(vb);
            const bool img = eo_candidate(vb) && vb.opsEO[0] != nullptr && vb.D1EO != nullptr && vb.D2EO != nullptr;
            par_ok = par_ok && img && vb.d2tc && eo_ok(vb, false);
            ff_ok = ff_ok && img;
            seo_ok = seo_ok && step_eo_candidate(vb) && vb.opsEO[0] != nullptr && vb.D1EO != nullptr;
        }
        if ((choice == 2 && !dnsk::helm_tc_supported(v0)) || (choice == 4 && !dnsk::spec_supported(v0)) ||
            (choice == 5 && !fuse_ok) || (choice == 6 && !par_ok) || (choice == 7 && !ff_ok) ||
            (choice == 8 && !seo_ok) || choice == 3)
            choice = 0;
        float t_choice = 0.f, t_sbs = 0.f;
        if (!choice) {
            float best[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int cand = 1; cand <= 8 && !rc; ++cand) {
                if (cand == 3 || (cand == 2 && !dnsk::helm_tc_supported(v0)) ||
                    (cand == 4 && !dnsk::spec_supported(v0)) || (cand == 5 && !fuse_ok) || (cand == 6 && !par_ok) ||
                    (cand == 7 && !ff_ok) || (cand == 8 && !seo_ok))
                    continue;
                for (const auto& P : h->parts[gi]) {
                    GroupView& vb = h->groups[P.ig].v;
                    vb.helm = cand == 8 ? 1 : cand >= 4 ? 4 : cand;
                    vb.d2fuse = cand == 5 ? 1 : 0;
                    vb.spec_eo = (cand == 6 || cand == 7) ? 1 : 0;
                    vb.spec_eoff = cand == 7 ? 1 : 0;
                    vb.step_eo = cand == 8 ? 1 : 0;
                }
                for (int w = 0; w < 2; ++w) enqueue_step(h);
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) enqueue_step(h);
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune per-wavenumber stage");
                if (!rc) cudaEventElapsedTime(&best[cand], e0, e1);
                best[cand] /= 3.f;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->launches = 0;
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            choice = 0;
            for (int cand = 1; cand <= 8; ++cand)
                if (best[cand] > 0.f && (choice == 0 || best[cand] < best[choice])) choice = cand;
            cache_store(h->cfg.autotune_cache, key, choice, best, 8);
            t_choice = best[choice];
            t_sbs = best[8];
        } else if (decided_t.count(key)) {
            t_choice = decided_t[key].first;
            t_sbs = decided_t[key].second;
        } else {
            t_choice = cache_lookup_time(h->cfg.autotune_cache, key, choice);
            t_sbs = cache_lookup_time(h->cfg.autotune_cache, key, 8);
        }
        decided[key] = choice;
        decided_t[key] = {t_choice, t_sbs};
        for (const auto& P : h->parts[gi]) {
            GroupView& v = h->groups[P.ig].v;
            v.helm = choice == 8 ? 1 : choice >= 4 ? 4 : choice;
            v.d2fuse = choice == 5 ? 1 : 0;
            v.spec_eo = (choice == 6 || choice == 7) ? 1 : 0;
            v.spec_eoff = choice == 7 ? 1 : 0;
            v.step_eo = choice == 8 ? 1 : 0;
            h->groups[P.ig].ygemm_sbs = v.ygemm;
            h->groups[P.ig].t_fused = t_choice;
            h->groups[P.ig].t_sbs = t_sbs;
            if (v.helm == 4) v.ygemm = 1;
        }
    }
    // linear groups: the apply kernels alone
    for (auto& G : h->groups) {
        GroupView& v = G.v;
        if (v.helm != 0) continue;
        const std::string key = tune_helm_key(v);
        int choice = decided.count(key) ? decided[key] : cache_lookup(h->cfg.autotune_cache, key);
        if ((choice == 2 && !dnsk::helm_tc_supported(v)) || (choice == 4 && (v.lin || !dnsk::spec_supported(v))) || choice == 3)
            choice = 0;
        if (!choice) {
            // the implicit apply is timed on sub-step 2 (both accumulators); it
            // writes only the sub-step state, which set_state overwrites later
            float best[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            // the persistent variant (3) fills the whole GPU, which timed alone
            // wins but inside the step starves the concurrent member blocks and
            // groups: only on request, never autotuned.  A DNS group times the
            // whole per-wavenumber part of a sub-step: the y-derivatives, the
            // forcing and the apply (1, 2) against the fused stage (4).
            const bool whole = !v.lin;
            for (int cand = 1; cand <= 4; ++cand) {
                if (cand == 2 && !dnsk::helm_tc_supported(v)) continue;
                if (cand == 3) continue;
                if (cand == 4 && !(whole && dnsk::spec_supported(v))) continue;
                auto run = [&]() {
                    if (cand == 4) {
                        dnsk::launch_spec(v, 1, st);
                        if (v.d2tc && !v.d2fuse) dnsk::launch_d2v_tc(v, v.v_s, st);
                        return;
                    }
                    if (whole) {
                        if (v.ygemm == 2) dnsk::launch_yderiv_tc(v, v.v_t, v.e_t, st);
                        else if (v.ygemm == 3) dnsk::launch_yderiv_eo(v, v.v_t, v.e_t, st);
                        else dnsk::launch_yderiv_t(v, v.v_t, v.e_t, st);
                        dnsk::launch_forcing_t(v, 1, st);
                    }
                    if (cand == 2) dnsk::launch_helm_tc(v, 1, st);
                    else dnsk::launch_helm_t(v, 1, st);
                };
                for (int w = 0; w < 2; ++w) run();
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5; ++r) run();
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune helm");
                if (rc) break;
                cudaEventElapsedTime(&best[cand], e0, e1);
                best[cand] /= 5.f;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            choice = 0;
            for (int cand = 1; cand <= 4; ++cand)
                if (best[cand] > 0.f && (choice == 0 || best[cand] < best[choice])) choice = cand;
            cache_store(h->cfg.autotune_cache, key, choice, best, 4);
        }
        decided[key] = choice;
        v.helm = choice;
        if (choice == 4) v.ygemm = 1;
    }
    // Tile shapes (neither changes a result: every column is computed the same
    // way whatever tile holds it).  Members per CTA of the fused stage:
    for (auto& G : h->groups) {
        GroupView& v = G.v;
        if (!precision_mixed(h) || v.helm != 4 || v.E < 2) continue;
        char kb[96];
        snprintf(kb, sizeof kb, "spec_ec %d %d %d %d", v.mx, v.my, v.mz, v.E);
        const std::string key = kb;
        std::vector<int> cands;
        const int ec_before = v.spec_ec;
        for (int ec : {std::min(v.E, 8), (std::min(v.E, 8) + 1) / 2, 2}) {
            v.spec_ec = ec;
            if (v.d2fuse && (ec > 4 || !dnsk::spec_d2fuse_supported(v))) continue;   // its N holds 4 members
            if (v.spec_eo && !dnsk::spec_eo_supported(v)) continue;
            if (ec >= 1 && dnsk::spec_supported(v) && std::find(cands.begin(), cands.end(), ec) == cands.end())
                cands.push_back(ec);
        }
        int choice = decided.count(key) ? decided[key] : cache_lookup_value(h->cfg.autotune_cache, key);
        if (std::find(cands.begin(), cands.end(), choice) == cands.end()) choice = 0;
        if (cands.empty()) {
            v.spec_ec = ec_before;
            continue;
        }
        if (!choice && cands.size() == 1) choice = cands[0];
        if (!choice) {
            std::vector<float> ms(cands.size(), 0.f);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
                v.spec_ec = cands[ci];
                for (int w = 0; w < 2; ++w) dnsk::launch_spec(v, 1, st);
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5; ++r) dnsk::launch_spec(v, 1, st);
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune fused-stage tile");
                if (!rc) cudaEventElapsedTime(&ms[ci], e0, e1);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            size_t best = 0;
            for (size_t ci = 1; ci < cands.size(); ++ci)
                if (ms[ci] < ms[best]) best = ci;
            choice = cands[best];
            for (auto& m : ms) m /= 5.f;
            cache_store_shape(h->cfg.autotune_cache, key, choice, cands, ms);
        }
        decided[key] = choice;
        v.spec_ec = choice;
    }
    // CTAs per SM of the fused stage in parity blocks (the registers budgeted
    // for 2 or for 3): by timing whole steps, every block of the group on the
    // candidate (a third CTA per SM helps the concurrent member blocks more
    // than it costs the kernel alone)
    for (size_t gi = 0; gi < h->parts.size(); ++gi) {
        GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
        if (!precision_mixed(h) || v0.helm != 4 || !v0.spec_eo) continue;
        char kb[96];
        snprintf(kb, sizeof kb, "spec_cta %d %d %d %d", v0.mx, v0.my, v0.mz, v0.E);
        const std::string key = kb;
        const std::vector<int> cands = {2, 3};
        int choice = decided.count(key) ? decided[key] : cache_lookup_value(h->cfg.autotune_cache, key);
        if (std::find(cands.begin(), cands.end(), choice) == cands.end()) choice = 0;
        if (!choice) {
            std::vector<float> ms(cands.size(), 0.f);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
                for (const auto& P : h->parts[gi]) h->groups[P.ig].v.spec_minb = cands[ci];
                for (int w = 0; w < 2; ++w) enqueue_step(h);
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) enqueue_step(h);
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune fused-stage CTAs per SM");
                if (!rc) cudaEventElapsedTime(&ms[ci], e0, e1);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->launches = 0;
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            size_t best = 0;
            for (size_t ci = 1; ci < cands.size(); ++ci)
                if (ms[ci] < ms[best]) best = ci;
            choice = cands[best];
            for (auto& m : ms) m /= 3.f;
            cache_store_shape(h->cfg.autotune_cache, key, choice, cands, ms);
        }
        decided[key] = choice;
        for (const auto& P : h->parts[gi]) h->groups[P.ig].v.spec_minb = choice;
    }
    // First column-tile cap of the register-tiled y-derivatives (in the
    // step-by-step stage every sub-step, with the fused stage for every newly
    // set state):
    for (auto& G : h->groups) {
        GroupView& v = G.v;
        if (!precision_mixed(h) || (v.ygemm != 1 && v.ygemm != 3)) continue;
        char kb[96];
        snprintf(kb, sizeof kb, "ytile %d %d %d %d", v.mx, v.my, v.mz, v.E);
        auto yd = [&]() {
            if (v.ygemm == 3) dnsk::launch_yderiv_eo(v, v.v_t, v.e_t, st);
            else dnsk::launch_yderiv_t(v, v.v_t, v.e_t, st);
        };
        const std::string key = kb;
        const std::vector<int> cands = {16, 32, 64};
        int choice = decided.count(key) ? decided[key] : cache_lookup_value(h->cfg.autotune_cache, key);
        if (std::find(cands.begin(), cands.end(), choice) == cands.end()) choice = 0;
        if (!choice) {
            std::vector<float> ms(cands.size(), 0.f);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
                v.yd_cap = cands[ci];
                for (int w = 0; w < 2; ++w) yd();
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5; ++r) yd();
                cudaEventRecord(e1, st);
                rc = check(h, cudaEventSynchronize(e1), "autotune y-derivative tile");
                if (!rc) cudaEventElapsedTime(&ms[ci], e0, e1);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            if ((rc = device_status(h))) return rc;
            size_t best = 0;
            for (size_t ci = 1; ci < cands.size(); ++ci)
                if (ms[ci] < ms[best]) best = ci;
            choice = cands[best];
            for (auto& m : ms) m /= 5.f;
            cache_store_shape(h->cfg.autotune_cache, key, choice, cands, ms);
        }
        decided[key] = choice;
        v.yd_cap = choice;
    }
    // the step-by-step stage in parity blocks for dns_advance's short calls, on
    // every block the autotuner put on the fused stage (not on a requested one)
    for (auto& G : h->groups) {
        G.has_sbs = false;
        G.p5_stale = false;
        const GroupView& v = G.v;
        if (!precision_mixed(h) || h->cfg.helm != 0 || v.lin || v.helm != 4) continue;
        GroupView a = v;
        a.helm = 1;
        a.d2fuse = 0;
        a.spec_eo = 0;
        a.spec_eoff = 0;
        a.step_eo = 1;
        a.ygemm = G.ygemm_sbs;
        const bool imgs = v.opsEO[0] != nullptr && v.opsEO[1] != nullptr && v.D1EO != nullptr &&
                          (a.ygemm != 3 || (v.D2EO != nullptr && v.D2lEO != nullptr)) &&
                          (a.ygemm != 2 || v.Atc != nullptr);
        if (!imgs || !dnsk::step_eo_supported(a) || (a.ygemm == 3 && !dnsk::yderiv_eo_supported(a))) continue;
        if (!(G.t_fused > 0.f && G.t_sbs > 0.f)) continue;   // no whole-step times for this group
        G.vsbs = a;
        G.has_sbs = true;
    }
    // what a short call saves on such a group: the derivatives of its uploaded
    // state (every block's, back to back), timed here on the workspace's contents
    for (size_t gi = 0; gi < h->parts.size() && !rc; ++gi) {
        if (!h->groups[h->parts[gi][0].ig].has_sbs) continue;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        auto derivs = [&]() {
            for (const auto& P : h->parts[gi])
                if (!rc) rc = new_state_derivatives(h, h->groups[P.ig].v, st);
        };
        derivs();
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) derivs();
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (!rc) rc = check(h, cudaEventSynchronize(e1), "time the derivatives of a new state");
        if (!rc) cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (const auto& P : h->parts[gi]) h->groups[P.ig].t_derivs = ms / 3.f;
    }
    h->launches = 0;
    if (rc) return rc;
    if ((rc = device_status(h))) return rc;
    h->bound = true;
    return DNS_OK;
}

int dns_state_shape(const dns_handle* h, int group, int* n_kx, int* n_kz, int* ny_int, int* my) {
    if (!h || group < 0 || group >= (int)h->parts.size()) return DNS_ERR_INVALID;
    const GroupView& v = h->groups[h->parts[group][0].ig].v;
    if (n_kx) *n_kx = v.nkx;
    if (n_kz) *n_kz = v.nkz;
    if (ny_int) *ny_int = v.ny;
    if (my) *my = v.my;
    return DNS_OK;
}

// True when the whole host range [p, p + bytes) is page-locked memory mapped
// into the device's address space at the same address (unified addressing), so
// that a kernel may read or write it directly.  Both ends of the range are
// checked; anything else (pageable memory, a mapping at another address) takes
// the staged path.
static bool host_mapped(const void* p, size_t bytes) {
    if (!p || bytes == 0) return false;
    const char* c = (const char*)p;
    const char* ends[2] = {c, c + bytes - 1};
    for (const char* q : ends) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer != (const void*)q) return false;
    }
    return true;
}

// The pack and unpack kernels move v, eta as 16-byte complex values and U, W as
// doubles: a caller's buffer is accessed by them only when so aligned.
static bool aligned_for_kernels(const void* v, const void* e, const void* U, const void* W) {
    return ((uintptr_t)v % 16) == 0 && ((uintptr_t)e % 16) == 0 && ((uintptr_t)U % 8) == 0 && ((uintptr_t)W % 8) == 0;
}

// After the pack kernel: a group on the fused stage keeps the y-derivatives of
// its state at time t in the per-plane arrays (every fused launch writes those
// of the state it produces), so a newly set state gets them here: in parity
// blocks as that stage computes them, else from the register-tiled kernel.
static int new_state_derivatives(dns_handle* h, const GroupView& v, cudaStream_t st) {
    int rc = check(h, cudaGetLastError(), "pack state");
    if (rc || !precision_mixed(h) || v.helm != 4) return rc;
    if (v.spec_eo) {
        dnsk::launch_eo_derivs(v, st);
        h->launches += 1;
        if (!v.spec_eoff) {
            dnsk::launch_d2v_tc(v, v.v_t, st);
            h->launches += 1;
        }
    } else {
        dnsk::launch_yderiv_t(v, v.v_t, v.e_t, st);
        h->launches += 1;
    }
    return check(h, cudaGetLastError(), "derivatives of the new state");
}

// direct: the sources are device memory or mapped host memory and the pack
// kernel reads them itself; otherwise they are copied (kind k) into the staging
// buffer (v, eta) and the profile rows (U, W) first.
static int set_state_block(dns_handle* h, int group, int member0, int count, const double* v_hat,
                           const double* eta_hat, const double* U00, const double* W00, bool direct,
                           cudaMemcpyKind k, cudaStream_t st) {
    GroupView& v = h->groups[group].v;
    if (member0 < 0 || count < 1 || member0 + count > v.E) return fail(h, DNS_ERR_INVALID, "member range");
    int rc;
    if (direct) {
        dnsk::launch_pack(v, member0, count, (const double2*)v_hat, (const double2*)eta_hat, v.lin ? nullptr : U00,
                          v.lin ? nullptr : W00, st);
        if (v.helm == 4) h->groups[group].p5_stale = false;
        return new_state_derivatives(h, v, st);
    }
    const size_t per = (size_t)count * v.ny * v.nmodes;
    if ((rc = check(h, cudaMemcpyAsync(v.stage, v_hat, per * sizeof(double2), k, st), "set v"))) return rc;
    if ((rc = check(h, cudaMemcpyAsync(v.stage + per, eta_hat, per * sizeof(double2), k, st), "set eta"))) return rc;
    if (!v.lin) {   // a linear group has no mean profiles (they stay zero)
        if ((rc = check(h, cudaMemcpyAsync(v.U_t + (size_t)member0 * v.my, U00, sizeof(double) * count * v.my, k, st),
                        "set U")))
            return rc;
        if ((rc = check(h, cudaMemcpyAsync(v.W_t + (size_t)member0 * v.my, W00, sizeof(double) * count * v.my, k, st),
                        "set W")))
            return rc;
    }
    dnsk::launch_pack(v, member0, count, v.stage, v.stage + per, nullptr, nullptr, st);
    if (v.helm == 4) h->groups[group].p5_stale = false;
    return new_state_derivatives(h, v, st);
}

int dns_set_state(dns_handle* h, int group, int member0, int count, const double* v_hat,
                  const double* eta_hat, const double* U00, const double* W00, int ptr_kind) {
    NvtxRange range_("dns_set_state");
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    if (ptr_kind != 0 && ptr_kind != 1) return fail(h, DNS_ERR_INVALID, "ptr_kind must be 0 or 1");
    const int E = h->descs[group].members;
    if (member0 < 0 || count < 1 || member0 + count > E) return fail(h, DNS_ERR_INVALID, "member range");
    const GroupView& v0 = h->groups[h->parts[group][0].ig].v;
    if (!v_hat || !eta_hat || (!v0.lin && (!U00 || !W00))) return fail(h, DNS_ERR_INVALID, "NULL state pointer");
    const size_t pm = (size_t)v0.ny * v0.nmodes * 2, pu = (size_t)v0.my;   // doubles per member
    const size_t bv = sizeof(double) * pm * count, bu = sizeof(double) * pu * count;
    const bool direct = aligned_for_kernels(v_hat, eta_hat, U00, W00) &&
                        (ptr_kind == 1 || (host_mapped(v_hat, bv) && host_mapped(eta_hat, bv) &&
                                           (v0.lin || (host_mapped(U00, bu) && host_mapped(W00, bu)))));
    const cudaMemcpyKind k = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (const auto& P : h->parts[group]) {
        const int lo = member0 > P.m0 ? member0 : P.m0;
        const int hi = (member0 + count) < (P.m0 + P.E) ? (member0 + count) : (P.m0 + P.E);
        if (lo >= hi) continue;
        const size_t o = (size_t)(lo - member0);
        int rc = set_state_block(h, P.ig, lo - P.m0, hi - lo, v_hat + o * pm, eta_hat + o * pm,
                                 U00 ? U00 + o * pu : nullptr, W00 ? W00 + o * pu : nullptr, direct, k, h->stream);
        if (rc) return rc;
    }
    // host buffers may be reused by the caller as soon as the call returns: one
    // synchronisation after every block's copies (or direct reads)
    if (ptr_kind == 0) return check(h, cudaStreamSynchronize(h->stream), "set state");
    return DNS_OK;
}

static int get_state_block(dns_handle* h, int group, int member0, int count, double* v_hat, double* eta_hat,
                           double* U00, double* W00, bool direct, cudaMemcpyKind k, cudaStream_t st) {
    GroupView& v = h->groups[group].v;
    if (member0 < 0 || count < 1 || member0 + count > v.E) return fail(h, DNS_ERR_INVALID, "member range");
    if (direct) {
        dnsk::launch_unpack(v, member0, count, (double2*)v_hat, (double2*)eta_hat, U00, W00, st);
        return check(h, cudaGetLastError(), "unpack state");
    }
    const size_t per = (size_t)count * v.ny * v.nmodes;
    dnsk::launch_unpack(v, member0, count, v.stage, v.stage + per, nullptr, nullptr, st);
    int rc;
    if ((rc = check(h, cudaGetLastError(), "unpack state"))) return rc;
    if (v_hat && (rc = check(h, cudaMemcpyAsync(v_hat, v.stage, per * sizeof(double2), k, st), "get v"))) return rc;
    if (eta_hat && (rc = check(h, cudaMemcpyAsync(eta_hat, v.stage + per, per * sizeof(double2), k, st), "get eta")))
        return rc;
    if (U00 && (rc = check(h, cudaMemcpyAsync(U00, v.U_t + (size_t)member0 * v.my, sizeof(double) * count * v.my, k, st),
                           "get U")))
        return rc;
    if (W00 && (rc = check(h, cudaMemcpyAsync(W00, v.W_t + (size_t)member0 * v.my, sizeof(double) * count * v.my, k, st),
                           "get W")))
        return rc;
    return DNS_OK;
}

int dns_get_state(const dns_handle* hc, int group, int member0, int count, double* v_hat,
                  double* eta_hat, double* U00, double* W00, int ptr_kind) {
    NvtxRange range_("dns_get_state");
    dns_handle* h = const_cast<dns_handle*>(hc);
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    if (ptr_kind != 0 && ptr_kind != 1) return fail(h, DNS_ERR_INVALID, "ptr_kind must be 0 or 1");
    const int E = h->descs[group].members;
    if (member0 < 0 || count < 1 || member0 + count > E) return fail(h, DNS_ERR_INVALID, "member range");
    const GroupView& v0 = h->groups[h->parts[group][0].ig].v;
    const size_t pm = (size_t)v0.ny * v0.nmodes * 2, pu = (size_t)v0.my;
    const size_t bv = sizeof(double) * pm * count, bu = sizeof(double) * pu * count;
    const bool direct = aligned_for_kernels(v_hat, eta_hat, U00, W00) &&
                        (ptr_kind == 1 || ((!v_hat || host_mapped(v_hat, bv)) && (!eta_hat || host_mapped(eta_hat, bv)) &&
                                           (!U00 || host_mapped(U00, bu)) && (!W00 || host_mapped(W00, bu))));
    const cudaMemcpyKind k = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (const auto& P : h->parts[group]) {
        const int lo = member0 > P.m0 ? member0 : P.m0;
        const int hi = (member0 + count) < (P.m0 + P.E) ? (member0 + count) : (P.m0 + P.E);
        if (lo >= hi) continue;
        const size_t o = (size_t)(lo - member0);
        int rc = get_state_block(h, P.ig, lo - P.m0, hi - lo, v_hat ? v_hat + o * pm : nullptr,
                                 eta_hat ? eta_hat + o * pm : nullptr, U00 ? U00 + o * pu : nullptr,
                                 W00 ? W00 + o * pu : nullptr, direct, k, h->stream);
        if (rc) return rc;
    }
    // one synchronisation after every block's unpack and copies
    return sync_with_status(h, h->stream, "get state");
}

// nsteps steps of every group on the handle's stream: the captured step graph
// (captured on first use) or the kernels enqueued directly; adds the launches
// to h->launches.
// The derivatives of the current state for every fused-stage block whose
// per-plane arrays a short dns_advance call left without them.
static int refresh_stale(dns_handle* h) {
    for (auto& G : h->groups) {
        if (!G.p5_stale) continue;
        G.p5_stale = false;
        int rc = new_state_derivatives(h, G.v, h->stream);
        if (rc) return rc;
    }
    return DNS_OK;
}

static int run_steps(dns_handle* h, int nsteps) {
    int rc;
    if (nsteps > 0 && (rc = refresh_stale(h))) return rc;
    if (h->cfg.use_graph) {
        if (h->stream == nullptr)
            return fail(h, DNS_ERR_INVALID, "graph capture needs a non-default stream (got the legacy NULL stream)");
        if (!h->gexec) {
            int before = h->launches;
            if ((rc = check(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
                return rc;
            enqueue_step(h);
            cudaGraph_t gr = nullptr;
            if ((rc = check(h, cudaStreamEndCapture(h->stream, &gr), "end capture"))) return rc;
            h->graph = gr;
            if ((rc = check(h, cudaGraphInstantiate(&h->gexec, gr, 0), "instantiate graph"))) return rc;
            h->graph_launches = h->launches - before;
            h->launches = before;
        }
        for (int i = 0; i < nsteps; ++i) {
            if ((rc = check(h, cudaGraphLaunch(h->gexec, h->stream), "graph launch"))) return rc;
            h->launches += h->graph_launches;
        }
    } else {
        for (int i = 0; i < nsteps; ++i) enqueue_step(h);
    }
    return check(h, cudaGetLastError(), "step launch");
}

int dns_step(dns_handle* h, int nsteps) {
    NvtxRange range_("dns_step");
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (nsteps < 0) return fail(h, DNS_ERR_INVALID, "nsteps < 0");
    h->launches = 0;
    return run_steps(h, nsteps);
}

// Upload, nsteps steps and download.  With direct transfers (device or mapped
// page-locked buffers) every member block runs on its own stream (pack, its
// sub-step kernels, unpack), the uploads one after another so that the first
// block computes while the next one's input is still crossing the link, and a
// block's download overlaps the blocks still computing; in graph mode the
// whole call is one captured graph, kept for the next call with the same
// buffers and step count.  Staged transfers (pageable memory, which a graph
// cannot hold) and long runs take the plain sequence: uploads, the step graph,
// downloads.  Per block the kernels and their order are those of
// dns_set_state + dns_step + dns_get_state, so the results are bitwise the same,
// except on a block the autotuner put on the fused stage in a call of at most
// ADVANCE_SBS_STEPS steps (captured whole, or eager) where the group's measured
// step-time gap over the call's steps is below what the derivatives of the
// uploaded state cost: that call runs the block's step-by-step stage in parity
// blocks, which needs none (the results are those of that stage, within the
// mixed step's budget of the fused one), and the next fused step of the block
// first computes the derivatives of its state.
int dns_advance(dns_handle* h, int nsteps, const dns_state_in* in, const dns_state_out* out, int ptr_kind) {
    NvtxRange range_("dns_advance");
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (nsteps < 0) return fail(h, DNS_ERR_INVALID, "nsteps < 0");
    if (ptr_kind != 0 && ptr_kind != 1) return fail(h, DNS_ERR_INVALID, "ptr_kind must be 0 or 1");
    const bool graph = h->cfg.use_graph != 0;
    if (graph && h->stream == nullptr)
        return fail(h, DNS_ERR_INVALID, "graph capture needs a non-default stream (got the legacy NULL stream)");
    const int ng = (int)h->parts.size();
    std::vector<char> din(ng, 0), dout(ng, 0);   // transfer path per group: direct or staged
    for (int gi = 0; gi < ng; ++gi) {
        const GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
        const size_t E = (size_t)h->descs[gi].members;
        const size_t bv = sizeof(double) * 2 * (size_t)v0.ny * v0.nmodes * E, bu = sizeof(double) * v0.my * E;
        if (in) {
            const dns_state_in& I = in[gi];
            if (!I.v_hat || !I.eta_hat || (!v0.lin && (!I.U00 || !I.W00)))
                return fail(h, DNS_ERR_INVALID, "group %d: NULL input pointer", gi);
            const double* U = v0.lin ? nullptr : I.U00;
            const double* W = v0.lin ? nullptr : I.W00;
            din[gi] = aligned_for_kernels(I.v_hat, I.eta_hat, U, W) &&
                      (ptr_kind == 1 || (host_mapped(I.v_hat, bv) && host_mapped(I.eta_hat, bv) &&
                                         (v0.lin || (host_mapped(U, bu) && host_mapped(W, bu)))));
        }
        if (out) {
            const dns_state_out& O = out[gi];
            dout[gi] = aligned_for_kernels(O.v_hat, O.eta_hat, O.U00, O.W00) &&
                       (ptr_kind == 1 || ((!O.v_hat || host_mapped(O.v_hat, bv)) &&
                                          (!O.eta_hat || host_mapped(O.eta_hat, bv)) &&
                                          (!O.U00 || host_mapped(O.U00, bu)) && (!O.W00 || host_mapped(O.W00, bu))));
        }
    }
    const bool multi = h->groups.size() > 1 && !h->gstreams.empty();
    auto bstream = [&](int ig) { return multi ? h->gstreams[ig] : h->stream; };
    int rc;
    for (auto& G : h->groups)
        if (!G.uploaded &&
            (rc = check(h, cudaEventCreateWithFlags(&G.uploaded, cudaEventDisableTiming), "upload event")))
            return rc;
    const cudaMemcpyKind kin = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    bool all_direct = true;
    for (int gi = 0; gi < ng; ++gi) all_direct = all_direct && (!in || din[gi]) && (!out || dout[gi]);
    const bool whole = graph && all_direct && nsteps <= ADVANCE_GRAPH_STEPS;   // one captured graph
    // short calls (captured whole, or eager) run a fused-stage block on its
    // step-by-step stage in parity blocks where the group's step-time gap over
    // the call's steps is below the derivatives of the uploaded state
    const bool sbs_window = nsteps <= ADVANCE_SBS_STEPS && (whole || !graph);
    auto alt = [&](const HostGroup& G) {
        return sbs_window && G.has_sbs && (float)nsteps * (G.t_sbs - G.t_fused) < G.t_derivs;
    };
    bool sbs = false;
    for (const auto& G : h->groups) sbs = sbs || alt(G);
    // a block's view swapped for its short-call one while its work is enqueued
    struct SbsView {
        HostGroup& G;
        bool on;
        SbsView(HostGroup& g, bool o) : G(g), on(o) { if (on) std::swap(G.v, G.vsbs); }
        ~SbsView() { if (on) std::swap(G.v, G.vsbs); }
    };
    // Fork, per block: upload (after the previous block's), nsteps steps,
    // download; join.
    auto enqueue_advance = [&]() -> int {
        int r;
        if (multi) cudaEventRecord(h->fork_ev, h->stream);
        cudaEvent_t prev_upload = nullptr;
        for (int gi = 0; gi < ng; ++gi) {
            const GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
            const size_t pm = (size_t)v0.ny * v0.nmodes * 2, pu = (size_t)v0.my;
            for (const auto& P : h->parts[gi]) {
                HostGroup& G = h->groups[P.ig];
                SbsView sw(G, alt(G));
                cudaStream_t sb = bstream(P.ig);
                const size_t o = (size_t)P.m0;
                if (multi) cudaStreamWaitEvent(sb, h->fork_ev, 0);
                if (in) {
                    const dns_state_in& I = in[gi];
                    if (prev_upload) cudaStreamWaitEvent(sb, prev_upload, 0);   // one upload at a time
                    if ((r = set_state_block(h, P.ig, 0, P.E, I.v_hat + o * pm, I.eta_hat + o * pm,
                                             I.U00 ? I.U00 + o * pu : nullptr, I.W00 ? I.W00 + o * pu : nullptr,
                                             din[gi] != 0, kin, sb)))
                        return r;
                    cudaEventRecord(G.uploaded, sb);
                    prev_upload = G.uploaded;
                    h->launches += 1;
                }
                for (int i = 0; i < nsteps; ++i) enqueue_group(h, G, sb, nullptr);
                if (out) {
                    const dns_state_out& O = out[gi];
                    if ((r = get_state_block(h, P.ig, 0, P.E, O.v_hat ? O.v_hat + o * pm : nullptr,
                                             O.eta_hat ? O.eta_hat + o * pm : nullptr,
                                             O.U00 ? O.U00 + o * pu : nullptr, O.W00 ? O.W00 + o * pu : nullptr,
                                             dout[gi] != 0, kout, sb)))
                        return r;
                    h->launches += 1;
                }
                if (multi) cudaEventRecord(h->gevents[P.ig], sb);
            }
        }
        if (multi)
            for (size_t ig = 0; ig < h->groups.size(); ++ig) cudaStreamWaitEvent(h->stream, h->gevents[ig], 0);
        return DNS_OK;
    };
    // a fused-stage block continuing its current state needs its derivatives
    if (!in)
        for (auto& G : h->groups) {
            if (!G.p5_stale || alt(G)) continue;
            G.p5_stale = false;
            if ((rc = new_state_derivatives(h, G.v, h->stream))) return rc;
        }
    if (whole) {
        // the whole call as one graph (one submission: every block starts at
        // once), kept for the next call with the same buffers and step count
        std::vector<uintptr_t> key = {(uintptr_t)nsteps, (uintptr_t)ptr_kind, (uintptr_t)(in != nullptr),
                                      (uintptr_t)(out != nullptr), (uintptr_t)sbs};
        for (int gi = 0; gi < ng; ++gi) {
            if (in) for (const void* q : {in[gi].v_hat, in[gi].eta_hat, in[gi].U00, in[gi].W00}) key.push_back((uintptr_t)q);
            if (out) for (const void* q : {out[gi].v_hat, out[gi].eta_hat, out[gi].U00, out[gi].W00}) key.push_back((uintptr_t)q);
        }
        if (!h->aexec || key != h->akey) {
            if (h->aexec) { cudaGraphExecDestroy(h->aexec); h->aexec = nullptr; }
            if (h->agraph) { cudaGraphDestroy(h->agraph); h->agraph = nullptr; }
            h->launches = 0;
            if ((rc = check(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
                return rc;
            int rc_enq = enqueue_advance();
            cudaGraph_t gr = nullptr;
            rc = check(h, cudaStreamEndCapture(h->stream, &gr), "end capture");
            if (rc_enq) { if (gr) cudaGraphDestroy(gr); return rc_enq; }
            if (rc) return rc;
            h->agraph = gr;
            if ((rc = check(h, cudaGraphInstantiate(&h->aexec, gr, 0), "instantiate advance graph"))) return rc;
            h->akey = key;
            h->alaunches = h->launches;
        }
        if ((rc = check(h, cudaGraphLaunch(h->aexec, h->stream), "advance graph launch"))) return rc;
        h->launches = h->alaunches;
    } else if (!graph) {
        h->launches = 0;
        if ((rc = enqueue_advance())) return rc;
    } else {
        // staged transfers (pageable memory cannot be captured) or many steps:
        // uploads, the step graph, downloads, one after another on the stream
        h->launches = 0;
        for (int gi = 0; gi < ng; ++gi) {
            const GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
            const size_t pm = (size_t)v0.ny * v0.nmodes * 2, pu = (size_t)v0.my;
            for (const auto& P : h->parts[gi]) {
                if (!in) break;
                const dns_state_in& I = in[gi];
                const size_t o = (size_t)P.m0;
                if ((rc = set_state_block(h, P.ig, 0, P.E, I.v_hat + o * pm, I.eta_hat + o * pm,
                                          I.U00 ? I.U00 + o * pu : nullptr, I.W00 ? I.W00 + o * pu : nullptr,
                                          din[gi] != 0, kin, h->stream)))
                    return rc;
                h->launches += 1;
            }
        }
        if ((rc = run_steps(h, nsteps))) return rc;
        for (int gi = 0; gi < ng; ++gi) {
            const GroupView& v0 = h->groups[h->parts[gi][0].ig].v;
            const size_t pm = (size_t)v0.ny * v0.nmodes * 2, pu = (size_t)v0.my;
            for (const auto& P : h->parts[gi]) {
                if (!out) break;
                const dns_state_out& O = out[gi];
                const size_t o = (size_t)P.m0;
                if ((rc = get_state_block(h, P.ig, 0, P.E, O.v_hat ? O.v_hat + o * pm : nullptr,
                                          O.eta_hat ? O.eta_hat + o * pm : nullptr, O.U00 ? O.U00 + o * pu : nullptr,
                                          O.W00 ? O.W00 + o * pu : nullptr, dout[gi] != 0, kout, h->stream)))
                    return rc;
                h->launches += 1;
            }
        }
    }
    for (auto& G : h->groups) G.p5_stale = G.p5_stale || alt(G);
    if ((rc = check(h, cudaGetLastError(), "advance launch"))) return rc;
    return sync_with_status(h, h->stream, "advance");
}

int dns_step_timed(dns_handle* h, int nsteps, double* ms, int* launches) {
    if (!h || !ms || !launches) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (nsteps < 0) return fail(h, DNS_ERR_INVALID, "nsteps < 0");
    for (int c = 0; c < DNS_K_NCLASS; ++c) { ms[c] = 0.0; launches[c] = 0; }
    h->launches = 0;
    int rc = nsteps > 0 ? refresh_stale(h) : DNS_OK;
    if (rc) return rc;
    for (int i = 0; i < nsteps && rc == DNS_OK; ++i) {
        Timer tm;
        enqueue_step(h, &tm);
        rc = check(h, cudaStreamSynchronize(h->stream), "timed step");
        for (size_t k = 1; k < tm.ev.size() && rc == DNS_OK; ++k) {
            if (tm.cls[k] < 0) continue;
            float t = 0.f;
            rc = check(h, cudaEventElapsedTime(&t, tm.ev[k - 1], tm.ev[k]), "event time");
            ms[tm.cls[k]] += t;
            launches[tm.cls[k]] += 1;
        }
        for (auto e : tm.ev) cudaEventDestroy(e);
    }
    if (rc) return rc;
    return check(h, cudaGetLastError(), "timed step launch");
}

// per-member statistics of one member block into per_member[0 .. E)
static int stats_block(dns_handle* h, int group, dns_stats_t* per_member, double* profiles) {
    GroupView& v = h->groups[group].v;
    cudaStream_t st = h->stream;
    dnsk::launch_stats(v, st);
    int rc;
    if ((rc = check(h, cudaGetLastError(), "stats launch"))) return rc;
    std::vector<double> out((size_t)v.E * 9);
    if ((rc = check(h, cudaMemcpyAsync(out.data(), v.st_out, out.size() * 8, cudaMemcpyDeviceToHost, st), "stats copy")))
        return rc;
    if (profiles &&
        (rc = check(h, cudaMemcpyAsync(profiles, v.prof, sizeof(double) * (size_t)v.E * 6 * v.my, cudaMemcpyDeviceToHost, st),
                    "profile copy")))
        return rc;
    if ((rc = sync_with_status(h, st, "stats"))) return rc;
    for (int e = 0; e < v.E; ++e) {
        dns_stats_t& s = per_member[e];
        const double* o = &out[(size_t)e * 9];
        s.e_total = o[0]; s.e_pert = o[1]; s.tau_bottom = o[2]; s.tau_top = o[3];
        s.bulk_flux = o[4]; s.gamma = o[5]; s.max_div = o[6];
        s.nonfinite = o[7] != 0.0 ? 1 : 0;
        s.cfl = o[8];
        s.reserved = 0;
    }
    return DNS_OK;
}

int dns_stats(dns_handle* h, int group, dns_stats_t* per_member, dns_stats_t* ensemble_mean, double* profiles) {
    NvtxRange range_("dns_stats");
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    if (!per_member) return fail(h, DNS_ERR_INVALID, "per_member is NULL");
    const int E = h->descs[group].members;
    const int my = h->groups[h->parts[group][0].ig].v.my;
    for (const auto& P : h->parts[group]) {
        int rc = stats_block(h, P.ig, per_member + P.m0, profiles ? profiles + (size_t)P.m0 * 6 * my : nullptr);
        if (rc) return rc;
    }
    bool any_nf = false;
    dns_stats_t mean;
    memset(&mean, 0, sizeof mean);
    for (int e = 0; e < E; ++e) {
        const dns_stats_t& s = per_member[e];
        any_nf = any_nf || s.nonfinite;
        mean.e_total += s.e_total / E; mean.e_pert += s.e_pert / E;
        mean.tau_bottom += s.tau_bottom / E; mean.tau_top += s.tau_top / E;
        mean.bulk_flux += s.bulk_flux / E; mean.gamma += s.gamma / E;
        mean.max_div = mean.max_div > s.max_div ? mean.max_div : s.max_div;
        mean.cfl = mean.cfl > s.cfl ? mean.cfl : s.cfl;
        mean.nonfinite |= s.nonfinite;
    }
    if (ensemble_mean) *ensemble_mean = mean;
    return any_nf ? DNS_ERR_NONFINITE : DNS_OK;
}

int dns_stats_noalloc(dns_handle* h, int group, double* out_dev) {
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    if (!out_dev) return fail(h, DNS_ERR_INVALID, "out_dev is NULL");
    for (const auto& P : h->parts[group]) {
        const GroupView& v = h->groups[P.ig].v;
        const size_t need = (size_t)v.E * v.ny * 6;
        if (need > dnsk::noalloc_max_partials())
            return fail(h, DNS_ERR_INVALID,
                        "dns_stats_noalloc: group %d needs %zu partial sums (members x (My-2) x 6), the fixed array holds %zu",
                        group, need, dnsk::noalloc_max_partials());
    }
    double* scratch = nullptr;
    int rc = check(h, dnsk::noalloc_scratch(&scratch), "dns_stats_noalloc: scratch address");
    if (rc) return rc;
    // member blocks one after another on the handle's stream (they share the array)
    for (const auto& P : h->parts[group]) {
        dnsk::launch_stats_noalloc(h->groups[P.ig].v, scratch, out_dev + (size_t)P.m0 * 8, h->stream);
        if ((rc = check(h, cudaGetLastError(), "dns_stats_noalloc launch"))) return rc;
    }
    return DNS_OK;
}

// ---- linearised disturbance groups

// Base flow on the (My, Mz) grid -> the nine fields the linear plane stage
// reads, on the interior planes: B, d_y B, d_z B for B = U, V, W.  Each field
// is truncated to |m| <= Kz first (its products with the disturbances are then
// free of aliasing on the 3/2 grid); d_y is the collocation derivative D1 on
// all My nodes, d_z spectral.  Plain host DFTs with the library's twiddles.
static void base_fields(const HostGroup& G, const std::vector<double>* f, std::vector<double>& out) {
    const GroupView& v = G.v;
    const int My = v.my, Mz = v.mz, Kz = v.kz, Ny = v.ny, NM = v.nkz;
    const std::vector<double> tw = dnsb::twiddles(Mz);   // exp(-2 pi i t / Mz)
    out.assign((size_t)9 * Ny * Mz, 0.0);
    std::vector<double> val((size_t)My * Mz), dz((size_t)My * Mz), cr(NM), ci(NM);
    for (int c = 0; c < 3; ++c) {
        const std::vector<double>& F = f[c];
        for (int y = 0; y < My; ++y) {
            for (int mi = 0; mi < NM; ++mi) {
                const int m = mi - Kz;
                double ar = 0.0, ai = 0.0;
                for (int z = 0; z < Mz; ++z) {
                    const int t = (int)((((long long)m * z) % Mz + Mz) % Mz);
                    ar += F[(size_t)y * Mz + z] * tw[2 * t];
                    ai += F[(size_t)y * Mz + z] * tw[2 * t + 1];
                }
                cr[mi] = ar / Mz;
                ci[mi] = ai / Mz;
            }
            for (int z = 0; z < Mz; ++z) {
                double sv = 0.0, sd = 0.0;
                for (int mi = 0; mi < NM; ++mi) {
                    const int m = mi - Kz;
                    const int t = (int)((((long long)m * z) % Mz + Mz) % Mz);
                    // exp(+2 pi i m z / Mz) = conj of the forward twiddle
                    const double er = tw[2 * t], ei = -tw[2 * t + 1];
                    sv += cr[mi] * er - ci[mi] * ei;
                    // i kz c exp(...): real part -kz (c_r e_i + c_i e_r)
                    sd += -G.kzt[mi] * (cr[mi] * ei + ci[mi] * er);
                }
                val[(size_t)y * Mz + z] = sv;
                dz[(size_t)y * Mz + z] = sd;
            }
        }
        for (int y = 1; y < My - 1; ++y)
            for (int z = 0; z < Mz; ++z) {
                double dy = 0.0;
                for (int k = 0; k < My; ++k) dy += G.grid.D1[(size_t)y * My + k] * val[(size_t)k * Mz + z];
                const size_t o = (size_t)(y - 1) * Mz + z;
                out[(size_t)c * Ny * Mz + o] = val[(size_t)y * Mz + z];
                out[(size_t)(3 + c) * Ny * Mz + o] = dy;
                out[(size_t)(6 + c) * Ny * Mz + o] = dz[(size_t)y * Mz + z];
            }
    }
}

static int linear_group(dns_handle* h, int group, HostGroup** G) {
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    HostGroup& g = h->groups[h->parts[group][0].ig];
    if (!g.v.lin) return fail(h, DNS_ERR_INVALID, "group %d is not a linear group", group);
    *G = &g;
    return DNS_OK;
}

int dns_set_base_flow(dns_handle* h, int group, const double* U, const double* V, const double* W, int ptr_kind) {
    if (!h) return DNS_ERR_INVALID;
    HostGroup* G = nullptr;
    int rc = linear_group(h, group, &G);
    if (rc) return rc;
    if (!U || !V || !W) return fail(h, DNS_ERR_INVALID, "NULL base-flow pointer");
    if (ptr_kind != 0 && ptr_kind != 1) return fail(h, DNS_ERR_INVALID, "ptr_kind must be 0 or 1");
    GroupView& v = G->v;
    const size_t n = (size_t)v.my * v.mz;
    std::vector<double> f[3];
    const double* src[3] = {U, V, W};
    for (int c = 0; c < 3; ++c) {
        f[c].resize(n);
        if (ptr_kind == 1) {
            if ((rc = check(h, cudaMemcpyAsync(f[c].data(), src[c], n * 8, cudaMemcpyDeviceToHost, h->stream),
                            "read base flow")))
                return rc;
        } else {
            memcpy(f[c].data(), src[c], n * 8);
        }
    }
    if (ptr_kind == 1 && (rc = check(h, cudaStreamSynchronize(h->stream), "read base flow"))) return rc;
    for (int c = 0; c < 3; ++c)
        for (double x : f[c])
            if (!std::isfinite(x)) return fail(h, DNS_ERR_INVALID, "base flow holds a non-finite value");
    std::vector<double> b;
    base_fields(*G, f, b);
    if ((rc = check(h, cudaMemcpyAsync((void*)v.base, b.data(), b.size() * 8, cudaMemcpyHostToDevice, h->stream),
                    "upload base flow")))
        return rc;
    std::vector<float> bf;
    if (precision_mixed(h)) {
        bf.assign(b.begin(), b.end());
        if ((rc = check(h, cudaMemcpyAsync((void*)v.basef, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, h->stream),
                        "upload base flow")))
            return rc;
    }
    return check(h, cudaStreamSynchronize(h->stream), "set base flow");
}

int dns_set_direction(dns_handle* h, int group, int adjoint) {
    if (!h) return DNS_ERR_INVALID;
    if (group == -1) {
        if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
        for (auto& G : h->groups)
            if (G.v.lin) {
                int rc = check(h, cudaMemsetAsync(G.v.dir, adjoint ? 1 : 0, sizeof(int), h->stream), "set direction");
                if (rc) return rc;
            }
        return DNS_OK;
    }
    HostGroup* G = nullptr;
    int rc = linear_group(h, group, &G);
    if (rc) return rc;
    return check(h, cudaMemsetAsync(G->v.dir, adjoint ? 1 : 0, sizeof(int), h->stream), "set direction");
}

int dns_orthonormalize(dns_handle* h, int group, double* norms) {
    NvtxRange range_("dns_orthonormalize");
    if (!h) return DNS_ERR_INVALID;
    HostGroup* G = nullptr;
    int rc = linear_group(h, group, &G);
    if (rc) return rc;
    dnsk::launch_lin_orthonormalize(G->v, h->stream);
    if ((rc = check(h, cudaGetLastError(), "orthonormalize launch"))) return rc;
    if (!norms) return DNS_OK;
    if ((rc = check(h, cudaMemcpyAsync(norms, G->v.gsr, sizeof(double) * G->v.E, cudaMemcpyDeviceToHost, h->stream),
                    "read norms")))
        return rc;
    return sync_with_status(h, h->stream, "orthonormalize");
}

int dns_optimal_sweep(dns_handle* h, int nsteps, double* gains) {
    NvtxRange range_("dns_optimal_sweep");
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (nsteps < 1) return fail(h, DNS_ERR_INVALID, "nsteps < 1");
    for (auto& G : h->groups)
        if (!G.v.lin) return fail(h, DNS_ERR_INVALID, "dns_optimal_sweep needs every group to be linear");
    int rc;
    if ((rc = dns_set_direction(h, -1, 0))) return rc;
    if ((rc = dns_step(h, nsteps))) return rc;
    int launches = h->launches;
    if ((rc = dns_set_direction(h, -1, 1))) return rc;
    if ((rc = dns_step(h, nsteps))) return rc;
    launches += h->launches;
    if ((rc = dns_set_direction(h, -1, 0))) return rc;
    for (auto& G : h->groups) {
        launches += dnsk::launch_lin_orthonormalize(G.v, h->stream);
        if ((rc = check(h, cudaGetLastError(), "orthonormalize launch"))) return rc;
    }
    h->launches = launches;
    if (!gains) return DNS_OK;
    size_t off = 0;
    for (auto& G : h->groups) {
        if ((rc = check(h, cudaMemcpyAsync(gains + off, G.v.gsr, sizeof(double) * G.v.E, cudaMemcpyDeviceToHost,
                                           h->stream),
                        "read gains")))
            return rc;
        off += G.v.E;
    }
    return sync_with_status(h, h->stream, "optimal sweep");
}

// ---- stochastic forcing

// Root of f on (lo, hi), where f changes sign, by bisection to the last bit.
static double bisect(const std::function<double(double)>& f, double lo, double hi) {
    double flo = f(lo);
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if (fm == 0.0) return mid;
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return 0.5 * (lo + hi);
}

// Forcing structures of a group at kx index n, per kz: the J least-damped
// eigenfunctions of each block of the diffusion operator on (Delta v, eta),
// sampled at the interior nodes and scaled to unit energy (the statistics'
// inner product of one complex kx column), k^2 = kx^2 + kz^2:
//   v (d/dt Delta v = Delta Delta v / Re, v = Dv = 0): Stokes modes by increasing mu,
//     even cos(mu y)/cos(mu) - cosh(k y)/cosh(k), mu tan(mu) = -k tanh(k), mu in ((m - 1/2) pi, m pi),
//     odd  sin(mu y)/sin(mu) - sinh(k y)/sinh(k), mu cot(mu) = k coth(k),  mu in (m pi, (m + 1/2) pi),
//     decay rate (mu^2 + k^2) / Re;
//   eta (d/dt eta = Delta eta / Re, eta = 0): sin(j pi (y + 1) / 2), rate ((j pi / 2)^2 + k^2) / Re.
// f: [NKZ][2][J][Ny] structures, rhs: their right-hand-side terms (-Delta f_v
// for F, -f_eta for G), lam: [NKZ][2][J] eigenvalues.
static void forcing_structures(const HostGroup& G, int n, int J, std::vector<double>& f, std::vector<double>& rhs,
                               std::vector<double>& lam) {
    const GroupView& v = G.v;
    const int Ny = v.ny, NKZ = v.nkz;
    const double pi = 3.141592653589793;
    f.assign((size_t)NKZ * 2 * J * Ny, 0.0);
    rhs.assign(f.size(), 0.0);
    lam.assign((size_t)NKZ * 2 * J, 0.0);
    const double* w = G.grid.ccw.data() + 1;
    const double* yy = G.grid.y.data() + 1;
    std::vector<double> phi(Ny), dphi(Ny);
    const double kx = G.kxt[n];
    auto finish = [&](int mi, int b, int j, double k2, double l, bool vblock) {
        double e = 0.0;
        if (vblock) {
            for (int r = 0; r < Ny; ++r) {
                double d = 0.0;
                for (int c = 0; c < Ny; ++c) d += G.D1i[(size_t)r * Ny + c] * phi[c];
                dphi[r] = d;
            }
            double e0 = 0.0, e1 = 0.0;
            for (int r = 0; r < Ny; ++r) { e0 += w[r] * phi[r] * phi[r]; e1 += w[r] * dphi[r] * dphi[r]; }
            e = 0.25 * (e0 + e1 / k2);
        } else {
            for (int r = 0; r < Ny; ++r) e += w[r] * phi[r] * phi[r];
            e = 0.25 * e / k2;
        }
        const double sc = std::sqrt(e);
        const size_t o = (((size_t)mi * 2 + b) * J + j) * Ny;
        for (int r = 0; r < Ny; ++r) f[o + r] = phi[r] / sc;
        for (int r = 0; r < Ny; ++r) {
            if (vblock) {
                double d = 0.0;
                for (int c = 0; c < Ny; ++c) d += G.D2i[(size_t)r * Ny + c] * f[o + c];
                rhs[o + r] = -(d - k2 * f[o + r]);
            } else {
                rhs[o + r] = -f[o + r];
            }
        }
        lam[((size_t)mi * 2 + b) * J + j] = l;
    };
    for (int mi = 0; mi < NKZ; ++mi) {
        const double kz = G.kzt[mi], k2 = kx * kx + kz * kz, k = std::sqrt(k2);
        const double th = std::tanh(k), cth = k / std::tanh(k);
        int j = 0;
        for (int m = 1; j < J; ++m)
            for (int odd = 0; odd < 2 && j < J; ++odd, ++j) {
                double mu;
                if (odd) {
                    mu = bisect([&](double x) { return x * std::cos(x) - cth * std::sin(x); }, m * pi + 1e-12,
                                (m + 0.5) * pi - 1e-12);
                    for (int r = 0; r < Ny; ++r) phi[r] = std::sin(mu * yy[r]) / std::sin(mu) - std::sinh(k * yy[r]) / std::sinh(k);
                } else {
                    mu = bisect([&](double x) { return x * std::sin(x) + k * th * std::cos(x); }, (m - 0.5) * pi + 1e-12,
                                m * pi - 1e-12);
                    for (int r = 0; r < Ny; ++r) phi[r] = std::cos(mu * yy[r]) / std::cos(mu) - std::cosh(k * yy[r]) / std::cosh(k);
                }
                finish(mi, 0, j, k2, -(mu * mu + k2) / v.re, true);
            }
        for (j = 0; j < J; ++j) {
            const double a = 0.5 * (j + 1) * pi;
            for (int r = 0; r < Ny; ++r) phi[r] = std::sin(a * (yy[r] + 1.0));
            finish(mi, 1, j, k2, -(a * a + k2) / v.re, false);
        }
    }
}

int dns_set_stochastic_forcing(dns_handle* h, int group, int kx_index, int n_eig, double rate, unsigned long long seed) {
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    const HostGroup& G0 = h->groups[h->parts[group][0].ig];
    if (G0.v.lin) return fail(h, DNS_ERR_INVALID, "group %d is linear: no stochastic forcing", group);
    if (!(rate >= 0.0) || !std::isfinite(rate)) return fail(h, DNS_ERR_INVALID, "rate must be finite and >= 0");
    const bool on = rate > 0.0;
    if (on && (kx_index < 1 || kx_index > G0.v.kx))
        return fail(h, DNS_ERR_INVALID, "kx_index must be in 1..Kx = %d", G0.v.kx);
    if (on && (n_eig < 1 || n_eig > dnsk::STOCH_NEIG_MAX || n_eig > G0.v.ny / 2))
        return fail(h, DNS_ERR_INVALID, "n_eig must be in 1..%d", std::min(dnsk::STOCH_NEIG_MAX, G0.v.ny / 2));
    std::vector<double> f, rhs, lam;
    if (on) forcing_structures(G0, kx_index, n_eig, f, rhs, lam);
    const double eps = on ? std::sqrt(rate / (2.0 * G0.v.nkz * 2 * n_eig)) : 0.0;
    int rc;
    for (const auto& P : h->parts[group]) {
        HostGroup& G = h->groups[P.ig];
        GroupView& v = G.v;
        v.fn = on ? kx_index : 0;
        v.fneig = on ? n_eig : 0;
        v.fscale = eps / std::sqrt(v.dt);
        v.fseed = seed;
        v.m0 = P.m0;
        v.Eu = h->descs[group].members;
        G.fstruct = f;
        G.flam = lam;
        if (!on) continue;
        if (!G.nstream) {
            if ((rc = check(h, cudaStreamCreateWithFlags(&G.nstream, cudaStreamNonBlocking), "noise stream"))) return rc;
            if ((rc = check(h, cudaEventCreateWithFlags(&G.nfork, cudaEventDisableTiming), "noise event"))) return rc;
            if ((rc = check(h, cudaEventCreateWithFlags(&G.njoin, cudaEventDisableTiming), "noise event"))) return rc;
        }
        if ((rc = check(h, cudaMemcpyAsync((void*)v.fbasis, rhs.data(), rhs.size() * 8, cudaMemcpyHostToDevice, h->stream),
                        "upload forcing structures")))
            return rc;
        if ((rc = check(h, cudaMemsetAsync(v.fstep, 0, sizeof(unsigned long long), h->stream), "reset noise step")))
            return rc;
    }
    // a captured step graph holds the previous group views
    drop_graphs(h);
    return check(h, cudaStreamSynchronize(h->stream), "set stochastic forcing");
}

int dns_export_forcing(const dns_handle* hc, int group, int m_index, double* structures, double* decay) {
    dns_handle* h = const_cast<dns_handle*>(hc);
    if (!h) return DNS_ERR_INVALID;
    if (group < 0 || group >= (int)h->parts.size()) return fail(h, DNS_ERR_INVALID, "bad group");
    const HostGroup& G = h->groups[h->parts[group][0].ig];
    if (G.v.fn <= 0) return fail(h, DNS_ERR_INVALID, "group %d has no stochastic forcing", group);
    if (m_index < 0 || m_index >= G.v.nkz) return fail(h, DNS_ERR_INVALID, "m_index out of range");
    const int J = G.v.fneig, Ny = G.v.ny;
    if (structures) memcpy(structures, &G.fstruct[(size_t)m_index * 2 * J * Ny], sizeof(double) * 2 * J * Ny);
    if (decay) memcpy(decay, &G.flam[(size_t)m_index * 2 * J], sizeof(double) * 2 * J);
    return DNS_OK;
}

int dns_selftest_timeout(dns_handle* h) {
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    dnsk::launch_wait_selftest(h->groups[0].v.status, h->stream);
    int rc = check(h, cudaGetLastError(), "selftest launch");
    if (rc) return rc;
    return sync_with_status(h, h->stream, "selftest");
}

int dns_selftest_bounds(dns_handle* h) {
    if (!h) return DNS_ERR_INVALID;
    if (!h->bound) return fail(h, DNS_ERR_INVALID, "workspace not bound");
    dnsk::launch_bounds_selftest(h->groups[0].v.status, h->stream);
    int rc = check(h, cudaGetLastError(), "selftest launch");
    if (rc) return rc;
    return sync_with_status(h, h->stream, "bounds selftest");
}

int dns_checked_build(void) {
#ifdef DNS_CHECK
    return 1;
#else
    return 0;
#endif
}

int dns_convert_selftest(const double* d_in, float* f_out, const float* f_in, double* d_out, long long n) {
    if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return DNS_ERR_INVALID;
    for (long long i = 0; i < n; ++i) {
        unsigned long long b;
        std::memcpy(&b, &d_in[i], 8);
        const unsigned fb = dnsk::d2f_bits((unsigned)(b >> 32), (unsigned)b);
        std::memcpy(&f_out[i], &fb, 4);
        unsigned fi, hi, lo;
        std::memcpy(&fi, &f_in[i], 4);
        dnsk::f2d_bits(fi, &hi, &lo);
        b = ((unsigned long long)hi << 32) | lo;
        std::memcpy(&d_out[i], &b, 8);
    }
    return DNS_OK;
}

int dns_destroy(dns_handle* h) {
    if (!h) return DNS_ERR_INVALID;
    if (h->bound) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (auto s2 : h->gstreams) cudaStreamDestroy(s2);
    for (auto& G : h->groups) {
        if (G.uploaded) cudaEventDestroy(G.uploaded);
        if (G.nstream) cudaStreamDestroy(G.nstream);
        if (G.nfork) cudaEventDestroy(G.nfork);
        if (G.njoin) cudaEventDestroy(G.njoin);
    }

    for (auto e2 : h->gevents) cudaEventDestroy(e2);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->hstatus) cudaFreeHost(h->hstatus);
    delete h;
    return DNS_OK;
}

const char* dns_last_error(const dns_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

int dns_kernel_choice(const dns_handle* h, int group, int* ygemm, int* plane, int* helm) {
    if (!h || group < 0 || group >= (int)h->parts.size()) return DNS_ERR_INVALID;
    const GroupView& v = h->groups[h->parts[group][0].ig].v;
    if (ygemm) *ygemm = v.ygemm;
    if (plane) *plane = v.plane;
    if (helm) *helm = v.helm == 1 && v.step_eo ? 8 : v.helm != 4 ? v.helm : v.d2fuse ? 5 : v.spec_eoff ? 7 : v.spec_eo ? 6 : 4;
    return DNS_OK;
}

int dns_last_launch_count(const dns_handle* h) { return h ? h->launches : 0; }

int dns_export_grid(const dns_handle* h, int group, double* y, double* D1, double* D2, double* D4c, double* ccw) {
    if (!h || group < 0 || group >= (int)h->parts.size()) return DNS_ERR_INVALID;
    const dnsb::GridOps& g = h->groups[h->parts[group][0].ig].grid;
    if (y) memcpy(y, g.y.data(), g.y.size() * 8);
    if (D1) memcpy(D1, g.D1.data(), g.D1.size() * 8);
    if (D2) memcpy(D2, g.D2.data(), g.D2.size() * 8);
    if (D4c) memcpy(D4c, g.D4c.data(), g.D4c.size() * 8);
    if (ccw) memcpy(ccw, g.ccw.data(), g.ccw.size() * 8);
    return DNS_OK;
}

int dns_export_operators(const dns_handle* h, int group, int h_index, int pair, double* Mv, double* Pv,
                         double* Me, double* Pe) {
    if (!h || group < 0 || group >= (int)h->parts.size() || h_index < 0 || h_index > 1) return DNS_ERR_INVALID;
    const HostGroup& G = h->groups[h->parts[group][0].ig];
    if (pair < 0 || pair >= G.v.npairs) return DNS_ERR_INVALID;
    const size_t nn = (size_t)G.v.ny * G.v.ny;
    const dnsb::CnOps& o = G.ops[h_index];
    if (Mv) memcpy(Mv, &o.Mv[pair * nn], nn * 8);
    if (Pv) memcpy(Pv, &o.Pv[pair * nn], nn * 8);
    if (Me) memcpy(Me, &o.Me[pair * nn], nn * 8);
    if (Pe) memcpy(Pe, &o.Pe[pair * nn], nn * 8);
    return DNS_OK;
}

}  // extern "C"
