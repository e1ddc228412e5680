#!/usr/bin/env python3
"""Throughput of the ensemble channel-DNS step on one node.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl gpu|reference] [--no-cpu-baseline] [--no-cpu-all-cores]

One step = one full CN/RK3 step (three sub-steps: y-derivatives, transforms and
advective products, forcing + RK combination, per-wavenumber implicit apply,
mean flow) for every member of the ensemble.  Workload: plane Poiseuille flow
at constant bulk flux, Re = 1650 (Re_tau ~ 100), box 2pi x 2 x pi, grid
64 x 65 x 64, 8 members, dt = 0.005, seeded 5% noise in |n|, |m| <= 4.

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank advances its
own independent ensemble (weak scaling, replicas: the step has no exchange
between members); only a barrier and a max of the per-rank times cross ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble member-steps/s (and grid-pts*steps/s) mixed vs FP64 on 1 GB300 at stated err"
UNIT = "member-steps/s"

# The default workload (the headline) and the other ensemble configurations.
WORKLOADS = {
    "couette16": dict(
        groups=[dict(flow="couette", mx=16, my=33, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01,
                     members=1)],
        name="Couette Re=400, 1.75pi x 2 x 1.2pi, 16x33x16, 1 member, dt=0.01 (laminar u = y + 1e-2 noise in "
             "|n|, |m| <= 2)",
        noise=[dict(seed0=1000, amp=1e-2, n_max=2, m_max=2)]),
    "poiseuille64": dict(
        groups=[dict(flow="poiseuille", mx=64, my=65, mz=64, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=8)],
        name="Poiseuille constant-flux Re=1650 (Re_tau~100), 2pi x 2 x pi, 64x65x64, 8 members, dt=0.005",
        noise=[dict(seed0=2000, amp=5e-2, n_max=4, m_max=4)]),
    "couette32": dict(
        groups=[dict(flow="couette", mx=32, my=49, mz=32, lx=1.75 * np.pi, lz=1.2 * np.pi, re=500.0, dt=0.01,
                     members=64)],
        name="Couette Re=500 (Re_tau~40 minimal box), 1.75pi x 2 x 1.2pi, 32x49x32, 64 members, dt=0.01",
        noise=[dict(seed0=3000, amp=5e-2, n_max=4, m_max=4)]),
    "uneven": dict(
        groups=[dict(flow="couette", mx=32, my=33, mz=32, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.005,
                     members=64),
                dict(flow="couette", mx=48, my=49, mz=48, lx=1.75 * np.pi, lz=1.2 * np.pi, re=800.0, dt=0.005,
                     members=32),
                dict(flow="poiseuille", mx=64, my=65, mz=64, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                     members=32)],
        name="uneven batch, 128 members in one graph: 64 x Couette 32x33x32 Re=400, 32 x Couette 48x49x48 Re=800, "
             "32 x Poiseuille 64x65x64 Re=1650, dt=0.005",
        noise=[dict(seed0=4000, amp=(1e-2, 5e-2), n_max=4, m_max=4), dict(seed0=4100, amp=(1e-2, 5e-2), n_max=4, m_max=4),
               dict(seed0=4200, amp=(1e-2, 5e-2), n_max=4, m_max=4)]),
    "rotational": dict(
        groups=[dict(flow="poiseuille", mx=64, my=65, mz=64, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=8,
                     form="rotational")],
        name="Poiseuille constant-flux Re=1650, 2pi x 2 x pi, 64x65x64, 8 members, dt=0.005, rotational nonlinear form",
        noise=[dict(seed0=2000, amp=5e-2, n_max=4, m_max=4)]),
    "s3t": dict(
        groups=[dict(flow="couette", mx=64, my=63, mz=64, lx=2 * np.pi, lz=1.2 * np.pi, re=1000.0, dt=0.01,
                     members=5, shared_mean=True)],
        name="shared-mean (S3T-type) Couette ensemble Re=1000, 2pi x 2 x 1.2pi, 64x63x64, 5 members, dt=0.01, "
             "stochastic forcing at kx/a = 1 (4 + 4 diffusion eigenfunctions per kz, e_pert injection 1e-5)",
        noise=[dict(seed0=6000, amp=2.5e-2, n_max=4, m_max=4)],
        forcing=[(1, 4, 1e-5, 6060)]),
    "channel128": dict(
        groups=[dict(flow="poiseuille", mx=128, my=97, mz=128, lx=4 * np.pi, lz=4 * np.pi / 3, re=3250.0, dt=0.002,
                     members=16)],
        name="Poiseuille constant-flux Re=3250 (Re_tau~180), 4pi x 2 x 4pi/3, 128x97x128, 16 members, dt=0.002",
        noise=[dict(seed0=5000, amp=1e-1, spectrum="kolmogorov")]),
    "optimal": dict(
        groups=[dict(flow="couette", mx=0, my=63, mz=64, lx=2 * np.pi, lz=np.pi, re=3000.0, dt=0.04, members=45,
                     linear=True, kx_index=n) for n in (1, 2, 3)],
        name="optimal disturbances: forward/adjoint linearised ensembles about a streak+roll Couette mean flow, "
             "Re=3000, 2pi x 2 x pi, My=63, Mz=64, kx = 1, 2, 3 x 45 vectors, dt = 5 x 0.008, T_opt = 15",
        noise=[dict(seed0=7000 + 100 * n) for n in (1, 2, 3)],
        base=dict(seed=77, streak=0.3, roll=0.03), t_opt=15.0),
}
WORKLOAD = WORKLOADS["poiseuille64"]["groups"][0]
WORKLOAD_NAME = WORKLOADS["poiseuille64"]["name"]
NOISE = WORKLOADS["poiseuille64"]["noise"][0]

FP32_PEAK_PER_SM_CLK = 128 * 2          # FP32 lanes x 2 flops (FMA) per SM per clock
FP64_NOMINAL_TFLOPS = 1.25              # GB300 FP64 (nominal)
ERR_HORIZON = 50                        # steps of the mixed-vs-FP64 error stated on the line


def initial_state(g, rank=0, noise=None):
    import dns_synth
    nz = dict(NOISE if noise is None else noise)
    if g.get("linear"):
        # disturbance vectors of one kx (no mean profiles)
        return dns_synth.make_disturbances(g["my"], g["mz"], g["lz"], g["members"], nz["seed0"] + 1000 * rank)
    amp = nz.get("amp", 5e-2)
    if isinstance(amp, tuple):     # amplitude ramp across members
        amp = np.linspace(amp[0], amp[1], g["members"])
    st = dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"],
                              nz["seed0"] + 1000 * rank, amp, n_max=nz.get("n_max"), m_max=nz.get("m_max"),
                              spectrum=nz.get("spectrum", "flat"))
    if g.get("shared_mean"):
        # members of a shared-mean ensemble start from one kx = 0 flow
        for k in ("v", "eta"):
            st[k][:, :, :, 0] = st[k][:, :, :, 0].mean(axis=0)[None]
        for k in ("U", "W"):
            st[k][:] = st[k].mean(axis=0)[None]
    return st


# ----------------------------------------------------------- distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, dist


def reduce_max(value, dist, device=None):
    """Max of a float over ranks (host plumbing only)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(member_steps_per_rank, seconds_per_rank, world):
    """Whole-job throughput: all ranks' member-steps over the slowest rank's time."""
    return member_steps_per_rank * world / seconds_per_rank


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- roofline

def kernel_work(cls, g, precision):
    """Algorithmic work of ONE launch of kernel class `cls` for group g:
    (bound, amount, unit).  Counts per unit are in the design notes."""
    ny, E = g["my"] - 2, g["members"]
    nkx = 1 if g.get("linear") else (g["mx"] - 1) // 3 + 1
    nkz = 2 * ((g["mz"] - 1) // 3) + 1
    nmodes = nkx * nkz
    S = nmodes * ny * E                      # complex values of one spectral field
    MM = g["mx"] * g["mz"]
    if cls == "plane" and g.get("linear"):
        # 9 inverse + 3 forward complex transforms of length Mz (5 N log2 N each),
        # the base-flow products (about 60 flops per z point)
        Mz = g["mz"]
        return "alu", E * ny * (12 * 5 * Mz * np.log2(Mz) + 60 * Mz), "flop"
    if cls == "plane":
        if g.get("form", "advective") == "rotational":
            # 6 inverse + 3 forward transforms, 6 products, the means
            per_plane = 9 * 2.5 * MM * np.log2(MM) + 6 * 2 * MM + 2 * 2 * MM
        else:
            # 12 inverse + 3 forward transforms, 9 products, the means
            per_plane = 15 * 2.5 * MM * np.log2(MM) + 9 * 2 * MM + 2 * 2 * MM
        return "alu", E * ny * per_plane, "flop"
    if cls == "yderiv":
        # in parity blocks ("simt_eo" y-derivatives) half the flops
        return "alu", S * 3 * 2 * 2 * ny * (0.5 if g.get("_ygemm") == "simt_eo" else 1.0), "flop"
    # the step-by-step forcing and apply in parity blocks ("simt_eo"): half the flops
    half = 0.5 if g.get("_stage") == "simt_eo" else 1.0
    if cls == "forcing":
        return "alu", S * 2 * 2 * ny * half, "flop"
    if cls == "helm":
        npairs = nkx * (nkz // 2 + 1)
        return "alu", 2 * npairs * 2 * 2 * ny * ny * 4 * E * half, "flop"
    if cls == "d2v":
        # D2 v of the new state: 2 ny flops per real output value
        return "alu", S * 2 * 2 * ny, "flop"
    if cls == "spec":
        # the fused stage: forcing (D1 phi), the implicit apply (M - I and P of
        # both fields; the third sub-step reuses (M_1 - I) x_t), the
        # y-derivatives of the new state (D2 v too where no separate kernel
        # computes it); 2 ny flops per output value of each
        npairs = nkx * (nkz // 2 + 1)
        apply = 2 * npairs * 2 * 2 * ny * ny * 4 * E * (5.0 / 6.0)
        work = S * 2 * 2 * ny * (4 if spec_computes_d2v(g) else 3) + apply
        # in parity blocks every product is two half-size blocks: half the flops
        return "alu", work / 2 if g.get("_stage") in ("fused_eo", "fused_eo_ff") else work, "flop"
    return "alu", E * 4.0 * (g["my"]) ** 2, "flop"


def spec_computes_d2v(g):
    """The fused stage writes D2 v itself: with the digit product inside it
    (per-wavenumber stage "fused_d2v"), in float-float (stage "fused_eo_ff", and
    above Ny = 64); else
    the separate tensor-core D2 v kernel does."""
    return g.get("_stage") in ("fused_d2v", "fused_eo_ff") or g["my"] - 2 > 64


def member_blocks(g):
    """Member blocks a group runs as (the library's rule: E/4 clamped to [4, 16],
    one block below 8 members, shared-mean and linear groups one block)."""
    if g.get("shared_mean") or g.get("linear"):
        return 1
    b = g.get("member_block", 0) or min(16, max(4, g["members"] // 4))
    return max(1, g["members"] // b)


def kernel_bytes(cls, g, precision):
    """Algorithmic DRAM bytes of kernel class `cls` over one sub-step of group g
    (every member): the arrays the kernel must read and write once, averaged
    over the three sub-steps where that differs.  Complex values: 8 B (FP32)
    or 16 B (FP64) in the P-layout and forcing arrays, 16 B in the FP64 state."""
    ny, E = g["my"] - 2, g["members"]
    nkx = 1 if g.get("linear") else (g["mx"] - 1) // 3 + 1
    nkz = 2 * ((g["mz"] - 1) // 3) + 1
    S = nkx * nkz * ny * E
    c = 8 if precision == "mixed" else 16
    if cls == "yderiv":
        return 2 * 16 * S + 5 * c * S                    # state in, 5 P-layout fields out
    if cls == "plane":
        return 5 * c * S + 3 * c * S                     # 5 fields in, 3 nonlinear terms out
    if cls == "forcing":
        return 3 * c * S + 2 * c * S + 2 * c * S * (4.0 / 3.0)   # N in, F G out, RK accumulators
    if cls == "d2v":
        return 16 * S + 8 * S                            # v (FP64) in, D2 v (P layout) out
    if cls == "spec":
        # N in (P layout), the state x_t in (first two sub-steps) and x+ out
        # (FP64), (M_1 - I) x_t out / in, the RK accumulators of F and G, the
        # operators (all four, two in the third sub-step), the P-layout fields
        # out (v, Dv, eta, D eta, and D2 v where this stage computes it)
        rp = (ny + 3) // 4 * 4
        npairs = nkx * (nkz // 2 + 1) - 1              # the mean mode's pair has no CTA
        # in parity blocks (per-wavenumber stage "fused_eo") a matrix is its even
        # and odd halves, ny x 2 ceil(ceil(ny / 2) / 2) floats
        mat = ny * 2 * (((ny + 1) // 2 + 1) // 2) if g.get("_stage") in ("fused_eo", "fused_eo_ff") else ny * rp
        ops = member_blocks(g) * npairs * ((4 + 4 + 2) / 3.0) * mat * 4
        state = 2 * S * (16 * (2.0 / 3.0) + 16 + 8 * (2.0 / 3.0))
        acc = 2 * 8 * S * (4.0 / 3.0)
        return ops + 3 * 8 * S + state + acc + (5 if spec_computes_d2v(g) else 4) * 8 * S
    if cls == "helm":
        rp = (ny + 3) // 4 * 4
        npairs = nkx * (nkz // 2 + 1)
        opb = 4 if precision == "mixed" else 8
        mats = (2 + 2 + 1) / 3.0                         # M and P, M reused in the third sub-step
        width = 2 * (((ny + 1) // 2 + 1) // 2) if g.get("_stage") == "simt_eo" else rp   # parity blocks
        ops = member_blocks(g) * npairs * 2 * mats * ny * (width if precision == "mixed" else ny) * opb
        m1 = (c if precision == "mixed" else 16) * (2.0 / 3.0)
        return ops + 2 * S * (16 * (2.0 / 3.0) + c + 16 + m1)   # x_t, F~ in, x+ out, M1 x_t
    return 0.0


def hbm_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def profiled_traffic(kernel, variant):
    """DRAM bytes per launch of kernel class `kernel` (variant `variant`) from
    the committed ncu record, or None when the record is of another variant or
    the kernel's sources changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_poiseuille64x65x64_E8_mixed.json")
    try:
        rec = json.load(open(path))["kernels"][kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("variant") != variant:
        return None
    h = hashlib.sha256()
    for f in rec["source_files"]:
        try:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            return None
    if h.hexdigest()[:16] != rec["source_sha256_16"]:
        return None
    return rec["dram_bytes_per_launch"]


def roofline_bound(flops, nbytes, alu_tflops, hbm_gbs):
    """'hbm' when the algorithmic intensity flops / nbytes lies below the ridge
    point alu peak / HBM peak (the memory roofline is the lower one), else 'alu'."""
    if nbytes <= 0:
        return "alu"
    ridge = alu_tflops * 1e12 / (hbm_gbs * 1e9)
    return "hbm" if flops / nbytes < ridge else "alu"


def alu_peak(precision_of_kernel, sm_mhz, n_sm):
    """FP32 peak of n_sm SMs at the sampled clock (TFLOP/s), or the nominal FP64
    rate."""
    if precision_of_kernel == "f64":
        return FP64_NOMINAL_TFLOPS
    return n_sm * FP32_PEAK_PER_SM_CLK * sm_mhz * 1e6 / 1e12


def rel_errors(got, ref):
    """Mixed-vs-FP64 relative errors of one group's states (v, eta, U, W as
    returned by get_state, U and W None for a linear group).  Per field and
    member: max |x - x_ref| / max |x_ref| over modes and y; the mean flow
    (U00, W00) is one velocity field normalised by max(|U00|, |W00|) of the
    reference, and W00 alone is reported on its own scale as well.  Returns the
    maxima over members and the per-member values."""
    E = ref[0].shape[0]
    out = {"v": [], "eta": [], "mean_flow": [], "w00_alone": []}
    for e in range(E):
        for k, i in (("v", 0), ("eta", 1)):
            a, b = np.asarray(got[i][e]), np.asarray(ref[i][e])
            out[k].append(float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)))
        if ref[2] is not None:
            du = np.abs(np.asarray(got[2][e]) - np.asarray(ref[2][e]))
            dw = np.abs(np.asarray(got[3][e]) - np.asarray(ref[3][e]))
            scale = max(np.max(np.abs(ref[2][e])), np.max(np.abs(ref[3][e])), 1e-300)
            out["mean_flow"].append(float(max(np.max(du), np.max(dw)) / scale))
            out["w00_alone"].append(float(np.max(dw) / max(np.max(np.abs(ref[3][e])), 1e-300)))
    res = {k: max(v) for k, v in out.items() if v}
    res["per_member"] = {k: v for k, v in out.items() if v}
    return res


def kernel_precision(cls, precision):
    # the mixed path runs every contraction and transform in FP32 (FP64 sums only)
    return "f64" if precision == "fp64" else "f32"


# ------------------------------------------------------------ cpu oracle

CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle, dns_synth
g = {g!r}
E = {members}
ch = oracle.Channel(g['mx'], g['my'], g['mz'], g['lx'], g['lz'], g['re'], g['dt'], g['flow'],
                    shared_mean=g.get('shared_mean', False), form=g.get('form', 'advective'))
if {forcing!r} is not None:
    from oracle.forcing import StochasticForcing
    ch.stochastic = StochasticForcing(ch, *{forcing!r})
st = dns_synth.make_state(g['mx'], g['my'], g['mz'], g['lx'], g['lz'], g['flow'], E, {seed0}, {amp},
                          n_max={n_max}, m_max={m_max})
x = tuple(st[k] for k in ('v', 'eta', 'U', 'W'))
for _ in range({warm}):
    x = ch.step(x, 1)
t = time.perf_counter()
for _ in range({steps}):
    x = ch.step(x, 1)
dt = time.perf_counter() - t
print(json.dumps(dict(seconds=dt, steps={steps}, members=E)))
"""


CPU_SNIPPET_LIN = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import dns_synth
from oracle.linear import Linear
g = {g!r}
E = {members}
b = dns_synth.make_base_flow(g['my'], g['mz'], g['lz'], g['flow'], {bseed}, streak={streak}, roll={roll})
lin = Linear(g['my'], g['mz'], g['lx'], g['lz'], g['re'], g['dt'], g['kx_index'], b['U'], b['V'], b['W'])
d = dns_synth.make_disturbances(g['my'], g['mz'], g['lz'], E, {seed0})
x = (d['v'], d['eta'])
for _ in range({warm}):
    x = lin.step(x, 1)
t = time.perf_counter()
for _ in range({steps}):
    x = lin.step(x, 1)
dt = time.perf_counter() - t
print(json.dumps(dict(seconds=dt, steps={steps}, members=E)))
"""


# All host cores: the oracle is built once (its operators in OpenMP), then one
# single-threaded worker per core is forked -- this process never touched CUDA
# -- and each advances its own member (members are independent); every worker
# warms up, waits at a barrier, and the rate is all members' steps over the
# time from the barrier to the last worker's end.
CPU_SNIPPET_PAR = r"""
import json, multiprocessing as mp, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import dns_synth
g = {g!r}
n = {nproc}
if g.get('linear'):
    from oracle.linear import Linear
    b = dns_synth.make_base_flow(g['my'], g['mz'], g['lz'], g['flow'], {bseed}, streak={streak}, roll={roll})
    ch = Linear(g['my'], g['mz'], g['lx'], g['lz'], g['re'], g['dt'], g['kx_index'], b['U'], b['V'], b['W'])
    def first(i):
        d = dns_synth.make_disturbances(g['my'], g['mz'], g['lz'], 1, {seed0} + i)
        return (d['v'], d['eta'])
else:
    import oracle
    ch = oracle.Channel(g['mx'], g['my'], g['mz'], g['lx'], g['lz'], g['re'], g['dt'], g['flow'],
                        shared_mean=g.get('shared_mean', False), form=g.get('form', 'advective'))
    if {forcing!r} is not None:
        from oracle.forcing import StochasticForcing
        ch.stochastic = StochasticForcing(ch, *{forcing!r})
    def first(i):
        st = dns_synth.make_state(g['mx'], g['my'], g['mz'], g['lx'], g['lz'], g['flow'], 1, {seed0} + i, {amp},
                                  n_max={n_max}, m_max={m_max})
        return tuple(st[k] for k in ('v', 'eta', 'U', 'W'))
ctx = mp.get_context('fork')
bar = ctx.Barrier(n + 1)
q = ctx.Queue()
def work(i):
    x = ch.step(first(i), 1)
    bar.wait()
    for _ in range({steps}):
        x = ch.step(x, 1)
    q.put(time.time())
ps = [ctx.Process(target=work, args=(i,)) for i in range(n)]
for p in ps:
    p.start()
bar.wait()
t0 = time.time()
ends = [q.get() for _ in range(n)]
for p in ps:
    p.join()
print(json.dumps(dict(seconds=max(ends) - t0, steps={steps}, members=n, workers=n)))
"""


def run_oracle_all_cores(g, nproc, steps, wl=None):
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    bw = (wl or {}).get("base", {"seed": 0, "streak": 0.0, "roll": 0.0})
    fc = None if g.get("linear") else (wl or {}).get("forcing", [None])[0]
    seed0 = wl["noise"][0]["seed0"] if g.get("linear") else NOISE["seed0"]
    code = CPU_SNIPPET_PAR.format(root=ROOT, g=g, nproc=nproc, bseed=bw["seed"], streak=bw["streak"],
                                  roll=bw["roll"], seed0=seed0, amp=NOISE["amp"], n_max=NOISE["n_max"],
                                  m_max=NOISE["m_max"], steps=steps, forcing=fc)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle(g, members, steps, warm=0, wl=None):
    env = dict(os.environ)
    # the timed steps run on one core (BLAS pinned to one thread, numpy's FFT is
    # single-threaded); only the untimed quad-precision operator build uses OpenMP
    for k in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    if g.get("linear"):
        bw = wl["base"]
        code = CPU_SNIPPET_LIN.format(root=ROOT, g=g, members=members, bseed=bw["seed"], streak=bw["streak"],
                                      roll=bw["roll"], seed0=wl["noise"][0]["seed0"], steps=steps, warm=warm)
    else:
        fc = (wl or {}).get("forcing", [None])[0]
        code = CPU_SNIPPET.format(root=ROOT, g=g, members=members, seed0=NOISE["seed0"], amp=NOISE["amp"],
                                  n_max=NOISE["n_max"], m_max=NOISE["m_max"], steps=steps, warm=warm, forcing=fc)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out


ARM_PARTS = {0xd4f: "Neoverse-V2", 0xd40: "Neoverse-V1", 0xd0c: "Neoverse-N1", 0xd49: "Neoverse-N2",
             0xd84: "Neoverse-V3"}


def cpu_info():
    """(model, logical cores).  Arm kernels list no model name: the implementer
    and part codes of /proc/cpuinfo name the core instead."""
    model, impl, part = "unknown", None, None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu model") and model == "unknown":
                    model = ln.split(":", 1)[1].strip()
                elif key == "cpu implementer" and impl is None:
                    impl = ln.split(":", 1)[1].strip()
                elif key == "cpu part" and part is None:
                    part = ln.split(":", 1)[1].strip()
    except OSError:
        pass
    if model == "unknown" and part is not None:
        try:
            name = ARM_PARTS.get(int(part, 16))
        except ValueError:
            name = None
        model = "Arm %s (implementer %s, part %s)" % (name or "core", impl, part)
    return model, os.cpu_count()


# ----------------------------------------------------------------- arms

def reference_arm(args, rank, world):
    if rank != 0:
        return
    g = WORKLOAD
    # each step a bounded sample of the workload: one member (the oracle advances
    # members independently, so member-steps/s does not depend on how many it
    # holds), at most 200 timed steps after at most 3 warm-up steps -- about a
    # minute of single-core numpy at 64x65x64, whatever --steps says
    n_steps, n_warm = max(1, min(args.steps, 200)), min(args.warmup, 3)
    out = run_oracle(g, 1, n_steps, warm=n_warm)
    value = out["members"] * out["steps"] / out["seconds"]
    model, ncpu = cpu_info()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * out["seconds"] / out["steps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded, dns_synth)",
        "config": {"workload": WORKLOAD_NAME, "precision": "fp64", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d steps x %d member of the workload (after %d warm-up steps; the run's --steps %d "
                                   "capped at 200), cpu %s, %d cores on host"
                                   % (out["steps"], out["members"], n_warm, args.steps, model, ncpu)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_arm(args, rank, world, dist):
    import torch
    import paper_2306_12739_gb300 as dns
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = WORKLOADS[args.workload]
    groups = [dict(g) for g in wl["groups"]]
    if args.member_block > 0:
        for g in groups:
            g["member_block"] = args.member_block
    states = [initial_state(g, rank, nz) for g, nz in zip(groups, wl["noise"])]
    members = sum(g["members"] for g in groups)
    # member grid points (a linear group's disturbance lives on the (y, z) plane of one harmonic)
    pts = sum(g["members"] * max(g["mx"], 1) * g["my"] * g["mz"] for g in groups)
    precision = args.precision
    linear = any(g.get("linear") for g in groups)
    if linear:
        import dns_synth
        bw = wl["base"]
        bases = [dns_synth.make_base_flow(g["my"], g["mz"], g["lz"], g["flow"], bw["seed"], streak=bw["streak"],
                                          roll=bw["roll"]) for g in groups]

    def load(ens):
        for gi, f in enumerate(wl.get("forcing", [])):
            if f is not None:
                ens.set_stochastic_forcing(gi, *f)
        for gi, st in enumerate(states):
            if groups[gi].get("linear"):
                ens.set_base_flow(gi, bases[gi]["U"], bases[gi]["V"], bases[gi]["W"])
                ens.set_state(gi, st["v"][..., None], st["eta"][..., None])
            else:
                ens.set_state(gi, st["v"], st["eta"], st["U"], st["W"])

    def timed_run(prec, nsteps, nwarm, flush):
        ens = dns.Ensemble(groups, precision=prec, use_graph=True, device=dev, ygemm=args.ygemm, plane=args.plane,
                           helm=args.helm)
        load(ens)
        stream = ens.stream
        ens.step(nwarm)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        launches = 0
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        with torch.cuda.stream(stream):
            for k in range(nsteps):
                flush.zero_()                  # evict L2 between timed steps
                starts[k].record(stream)
                ens.step(1)
                launches += ens.launches()
                ends[k].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if dist is not None:
            dist.barrier()
        total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        return ens, total_ms, launches, clocks

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ens, total_ms, launches, clocks = timed_run(precision, args.steps, args.warmup, flush)
    choices = [dict(ygemm=dns.dns_kernel_choice(ens.h, gi, "ygemm"), plane=dns.dns_kernel_choice(ens.h, gi, "plane"),
                    helm=dns.dns_kernel_choice(ens.h, gi, "helm")) for gi in range(len(groups))]
    for g, ch in zip(groups, choices):
        g["_stage"] = ch["helm"]            # the byte and flop models of the fused stage depend on it
        g["_ygemm"] = ch["ygemm"]
    total_ms = reduce_max(total_ms, dist, dev)
    ms_step = total_ms / args.steps
    value = aggregate(members * args.steps, total_ms / 1e3, world)

    # per-kernel device times (events around every launch), for the roofline
    load(ens)
    n_timed = max(1, min(args.steps, 5))
    kt = ens.step_timed(n_timed)
    tot = sum(v[0] for v in kt.values())
    kt = {k: v for k, v in kt.items() if v[1] > 0}          # classes that launched
    shares = {k: (v[0] / tot if tot > 0 else 0.0) for k, v in kt.items()}
    dom = max(kt, key=lambda k: kt[k][0])
    # every member of every group passes through the kernel once per sub-step
    # (member blocks split a group over several launches; the work is per member)
    work = sum(kernel_work(dom, g, precision)[1] for g in groups) * 3 * n_timed
    dbytes = sum(kernel_bytes(dom, g, precision) for g in groups) * 3 * n_timed
    avg_ms = kt[dom][0] / max(1, kt[dom][1])
    kprec = kernel_precision(dom, precision)
    sm_mhz = clocks["sm_mhz"] or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    hpk, hsrc = hbm_peak()
    apk = alu_peak(kprec, sm_mhz, n_sm)
    # the roofline that bounds the kernel at its algorithmic intensity: HBM below
    # the ridge (peak flops / peak bytes per second), the ALU peak above it
    bound = roofline_bound(work, dbytes, apk, hpk)
    if bound == "hbm":
        peak, unit = hpk, "GB/s"
        achieved = dbytes / (kt[dom][0] / 1e3) / 1e9
    else:
        peak, unit = apk, "TFLOP/s"
        achieved = work / (kt[dom][0] / 1e3) / 1e12
    variant = {"plane": choices[0]["plane"], "yderiv": choices[0]["ygemm"], "helm": choices[0]["helm"],
               "spec": choices[0]["helm"], "d2v": "tc"}.get(dom, "simt")
    traffic = (profiled_traffic(dom, variant)
               if (precision == "mixed" and args.workload == "poiseuille64") else None)
    # every class against the HBM roofline of its own algorithmic bytes (the
    # event pass runs the kernels one at a time)
    per_class = {}
    for cls, (ms, nl) in kt.items():
        b = sum(kernel_bytes(cls, g, precision) for g in groups) * 3 * n_timed
        if b <= 0 or ms <= 0:
            continue
        gbs = b / (ms / 1e3) / 1e9
        per_class[cls] = {"ms_per_launch": ms / max(1, nl), "algorithmic_bytes_per_launch": b / max(1, nl),
                          "achieved_gbs": gbs, "frac_of_hbm": gbs / hpk}
    roofline = {"kernel": dom, "bound": bound, "precision": kprec, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu, profiles/)",
                "intensity_flop_per_byte": work / dbytes if dbytes > 0 else None,
                "ridge_flop_per_byte": apk * 1e3 / hpk,
                "alu_peak_tflops": apk, "hbm_peak_gbs": hpk,
                "peak_source": (hsrc if bound == "hbm" else "nominal GB300 FP64" if kprec == "f64" else
                                "%d SM (device attribute) x 128 FP32 lanes x 2 x median sampled SM clock %.0f MHz"
                                % (n_sm, sm_mhz)),
                "kernel_ms_per_launch": avg_ms,
                "shares": {k: round(v, 4) for k, v in shares.items()},
                "hbm_view": {"peak_gbs": hpk, "peak_source": hsrc, "classes": per_class}}

    # the mixed states after ERR_HORIZON steps of this very launch configuration
    # (same handle, kernel variants, member blocks and graph), for the error
    # against FP64 stated on the line
    mixed_states = None
    if precision == "mixed" and not args.no_fp64:
        load(ens)
        ens.step(ERR_HORIZON)
        mixed_states = [ens.get_state(gi) for gi in range(len(groups))]

    # end to end through the C ABI with host buffers: upload state, step, download state
    pins, outs = [], []
    for st in states:
        keys = ("v", "eta") if "U" not in st else ("v", "eta", "U", "W")
        pin = [torch.from_numpy(np.ascontiguousarray(st[k]).view(np.float64)).pin_memory() for k in keys]
        pin += [None] * (4 - len(pin))
        pins.append(pin)
        outs.append([torch.empty_like(p).pin_memory() if p is not None else None for p in pin])
    h2d = sum(p.numel() * 8 for pin in pins for p in pin if p is not None)
    d2h = sum(o.numel() * 8 for out in outs for o in out if o is not None)
    ptr = lambda t: t.data_ptr() if t is not None else None
    e2e_steps = max(1, min(args.steps, 50))
    ins_p = [tuple(ptr(p) for p in pin) for pin in pins]
    outs_p = [tuple(ptr(o) for o in out) for out in outs]
    for _ in range(max(3, args.warmup)):   # the first call captures the member blocks' step graphs
        dns.dns_advance(ens.h, 1, ins_p, outs_p, 0)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        # one call per step: upload every group from page-locked memory, one
        # step, download (member blocks overlap transfers with computation)
        dns.dns_advance(ens.h, 1, ins_p, outs_p, 0)
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, dev)
    e2e_value = aggregate(members * e2e_steps, e2e_s, world)
    optimal = None
    if "t_opt" in wl:
        # one whole optimal-growth iteration of every group: T_opt forward, T_opt
        # adjoint, Gram-Schmidt (device time, L2 not flushed inside it)
        nopt = int(round(wl["t_opt"] / groups[0]["dt"]))
        load(ens)
        ens.optimal_sweep(nopt)                       # warm (graph already captured)
        load(ens)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ens.stream)
        gains = ens.optimal_sweep(nopt)
        e1.record(ens.stream)
        torch.cuda.synchronize()
        optimal = {"iteration_s": e0.elapsed_time(e1) / 1e3, "steps_each_way": nopt,
                   "vectors": members, "launches": ens.launches(),
                   "leading_gain_estimates": [float(np.max(gn)) for gn in gains]}
    ens.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if precision == "mixed" else "f64",
        "data": "synthetic (seeded, dns_synth)",
        "config": {"workload": wl["name"], "precision": precision, "graph": True,
                   "kernels": choices, "ygemm_request": args.ygemm, "plane_request": args.plane,
                   "helm_request": args.helm, "member_block_request": args.member_block,
                   "l2": "flushed (256 MiB write) before every timed step", "parallelism": "replicas x%d" % world},
        "grid_pts_steps_per_s": aggregate(pts * args.steps, total_ms / 1e3, world),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps,
                "call": "dns_advance per step: upload from page-locked host memory, one step, download"},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
    }
    if optimal is not None:
        line["optimal_iteration"] = optimal

    if precision == "mixed" and not args.no_fp64:
        n64 = max(20, min(args.steps, 50))
        ens64, t64, _, _ = timed_run("fp64", n64, min(args.warmup, 3), flush)
        load(ens64)
        ens64.step(ERR_HORIZON)
        errs = []
        for gi in range(len(groups)):
            st64 = ens64.get_state(gi)
            got = mixed_states[gi]
            if groups[gi].get("linear"):
                st64, got = (st64[0], st64[1], None, None), (got[0], got[1], None, None)
            errs.append(rel_errors(got, st64))
        ens64.close()
        t64 = reduce_max(t64, dist, dev)
        v64 = aggregate(members * n64, t64 / 1e3, world)
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": t64 / n64, "steps": n64}
        line["mixed_over_fp64"] = value / v64
        fields = [k for k in ("v", "eta", "mean_flow", "w00_alone") if k in errs[0]]
        line["err_vs_fp64"] = {
            "horizon_steps": ERR_HORIZON,
            "metric": "max over members of max|mixed - fp64| / max|fp64| per field, after the same seeded steps "
                      "(mean flow: U00 and W00 as one field; w00_alone on its own scale)",
            "max": {k: max(e[k] for e in errs if k in e) for k in fields},
            # the parity tests' bounds: DNS fields 1e-6 (W00 on its own scale 3e-5), linearised
            # disturbance vectors 1e-5 (their growth amplifies the single-precision rounding)
            "tolerance": ({"v": 1e-5, "eta": 1e-5} if any(g.get("linear") for g in groups) else
                          {"v": 1e-6, "eta": 1e-6, "mean_flow": 1e-6, "w00_alone": 3e-5}),
            "per_group": [{k: e[k] for k in fields if k in e} for e in errs],
            "per_member_first_group": errs[0]["per_member"],
        }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g0 = groups[0]
        if g0.get("linear"):
            out = run_oracle(g0, g0["members"], 10, wl=wl)     # about 7 s of single-core numpy
        else:
            out = run_oracle(g0, min(g0["members"], 4), 2, wl=wl)
        model, ncpu = cpu_info()
        line["cpu_baseline"] = {"value": out["members"] * out["steps"] / out["seconds"], "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": "%d steps x %d members of the workload's first group, single-threaded numpy, "
                                          "cpu %s (%d cores on host)" % (out["steps"], out["members"], model, ncpu)}
        if not args.no_cpu_all_cores:
            try:
                avail = len(os.sched_getaffinity(0))
            except AttributeError:
                avail = ncpu
            try:
                par = run_oracle_all_cores(g0, avail, 20 if g0.get("linear") else 2, wl=wl)
                line["cpu_baseline_all_cores"] = {
                    "value": par["members"] * par["steps"] / par["seconds"], "unit": UNIT, "cores": par["workers"],
                    "kind": "oracle",
                    "sample": "%d single-threaded oracle workers (forked after one operator build), one member of "
                              "the workload's first group each, %d steps after a barrier, cpu %s"
                              % (par["workers"], par["steps"], model)}
            except (RuntimeError, OSError, ValueError) as exc:   # a secondary figure: never lose the line for it
                line["cpu_baseline_all_cores"] = {"unavailable": str(exc).splitlines()[-1][:200] if str(exc) else
                                                  type(exc).__name__}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the oracle timing over all host cores (one forked worker per core)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator run")
    ap.add_argument("--plane", choices=["default", "cta", "cluster", "lines"], default="default",
                    help="plane-stage kernel (default: autotuned among those the grid supports)")
    ap.add_argument("--helm", choices=["default", "simt", "tc", "persist", "fused", "fused_d2v", "fused_eo", "fused_eo_ff", "simt_eo"], default="default",
                    help="per-wavenumber stage of the mixed path (default: the fused stage where the group "
                         "supports it, else the autotuned implicit apply)")
    ap.add_argument("--ygemm", choices=["default", "simt", "tc", "simt_eo"], default="default",
                    help="y-contraction variant of the mixed path")
    ap.add_argument("--member-block", type=int, default=0,
                    help="members per block of every independent-member group (0: the library's rule)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="poiseuille64",
                    help="ensemble configuration (default: the headline 64x65x64 Poiseuille ensemble)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, dist = dist_setup()
    if args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        gpu_arm(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
