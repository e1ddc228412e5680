"""Host logic of bench.py, on the CPU: the member-block rule it uses for its byte
model (the library's: E/4 clamped to [4, 16] members per block, the quotient
rounded down), the whole-job aggregate, the CPU name on Arm hosts, and the
oracle timing over all host cores (one forked single-threaded worker per
member)."""
import builtins
import io

import numpy as np
import pytest

import bench

G = dict(flow="couette", mx=16, my=17, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=2)


@pytest.mark.parametrize("members,block,blocks", [(1, 0, 1), (5, 0, 1), (7, 0, 1), (8, 0, 2), (12, 0, 3),
                                                  (16, 0, 4), (64, 0, 4), (128, 0, 8), (200, 0, 12),
                                                  (5, 2, 2), (6, 3, 2), (8, 4, 2), (3, 4, 1)])
def test_member_blocks_follow_the_library_rule(members, block, blocks):
    assert bench.member_blocks(dict(members=members, member_block=block)) == blocks


def test_shared_mean_and_linear_groups_are_one_block():
    assert bench.member_blocks(dict(members=64, shared_mean=True)) == 1
    assert bench.member_blocks(dict(members=45, linear=True)) == 1


def test_aggregate_counts_every_rank_against_the_slowest():
    assert bench.aggregate(800, 2.0, 1) == 400.0
    assert bench.aggregate(800, 2.0, 4) == 1600.0


def test_cpu_info_names_arm_cores(monkeypatch):
    text = ("processor\t: 0\nBogoMIPS\t: 2000.00\nFeatures\t: fp asimd\nCPU implementer\t: 0x41\n"
            "CPU architecture: 8\nCPU variant\t: 0x0\nCPU part\t: 0xd4f\nCPU revision\t: 0\n")
    real_open = builtins.open
    monkeypatch.setattr(builtins, "open",
                        lambda p, *a, **k: io.StringIO(text) if p == "/proc/cpuinfo" else real_open(p, *a, **k))
    model, n = bench.cpu_info()
    assert model == "Arm Neoverse-V2 (implementer 0x41, part 0xd4f)" and n >= 1


def test_oracle_on_all_cores_times_one_member_per_worker():
    out = bench.run_oracle_all_cores(G, 2, 2, wl=bench.WORKLOADS["poiseuille64"])
    assert out["workers"] == 2 and out["members"] == 2 and out["steps"] == 2
    assert 0.0 < out["seconds"] < 120.0


def test_byte_and_work_models_are_the_documented_counts():
    """The algorithmic bytes and flops that the roofline figures divide by, for
    one launch of the headline case (64x65x64, one member block of 4): S =
    modes x Ny x E complex values; y-derivatives 2*16 S in + 5*8 S out, plane
    stage 5*8 S in + 3*8 S out, forcing 3*8 S + 2*8 S + the RK accumulators
    (2*8 S, read in two sub-steps of three and written in all); the plane stage
    15 * 2.5 MxMz log2(MxMz) + 22 MxMz flop per plane and member."""
    g = dict(bench.WORKLOADS["poiseuille64"]["groups"][0], members=4)
    S = 22 * 43 * 63 * 4
    assert bench.kernel_bytes("yderiv", g, "mixed") == 72 * S == 17164224
    assert bench.kernel_bytes("plane", g, "mixed") == 64 * S == 15257088
    assert bench.kernel_bytes("forcing", g, "mixed") == pytest.approx((40 + 16 * 4 / 3) * S) == 14621376
    bound, flops, unit = bench.kernel_work("plane", g, "mixed")
    per = 15 * 2.5 * 4096 * 12 + 22 * 4096
    assert (bound, unit) == ("alu", "flop") and flops == pytest.approx(4 * 63 * per)
    # the fused stage: N in, the FP64 state, the RK accumulators, the operators of
    # 22 x 22 - 1 wavenumber pairs (4 + 4 + 2 matrices over three sub-steps; the
    # mean mode's pair has none), and four P-layout fields out, five when it
    # computes D2 v itself
    ops = 483 * (10 / 3) * 63 * 64 * 4
    base = ops + 24 * S + 2 * S * (16 * 2 / 3 + 16 + 8 * 2 / 3) + 16 * S * 4 / 3
    assert bench.kernel_bytes("spec", g, "mixed") == pytest.approx(base + 32 * S)
    assert bench.kernel_bytes("spec", dict(g, _stage="fused_d2v"), "mixed") == pytest.approx(base + 40 * S)
    _, w4, _ = bench.kernel_work("spec", g, "mixed")
    _, w5, _ = bench.kernel_work("spec", dict(g, _stage="fused_d2v"), "mixed")
    assert w5 - w4 == pytest.approx(S * 4 * 63)


def test_alu_peak_scales_with_the_sm_count_and_clock():
    assert bench.alu_peak("f32", 2070.0, 152) == pytest.approx(152 * 256 * 2.07e9 / 1e12)
    assert bench.alu_peak("f32", 1000.0, 100) == pytest.approx(100 * 256 * 1e9 / 1e12)
    assert bench.alu_peak("f64", 2070.0, 152) == bench.FP64_NOMINAL_TFLOPS


def test_rel_errors_per_field_and_member():
    rng = np.random.default_rng(3)
    E, ny, nkz, nkx, my = 3, 5, 7, 4, 7
    v = rng.standard_normal((E, ny, nkz, nkx)) + 1j * rng.standard_normal((E, ny, nkz, nkx))
    eta = 2.0 * v[::-1].copy()
    U = rng.standard_normal((E, my))
    W = 1e-3 * rng.standard_normal((E, my))
    ref = (v, eta, U, W)
    got = (v.copy(), eta.copy(), U.copy(), W.copy())
    got[0][1, 2, 3, 1] += 1e-7                        # member 1, v
    got[3][2, 4] += 1e-9                              # member 2, W00
    r = bench.rel_errors(got, ref)
    assert r["v"] == pytest.approx(1e-7 / np.max(np.abs(v[1])), rel=1e-6)
    assert r["per_member"]["v"][0] == 0.0 and r["per_member"]["v"][2] == 0.0
    assert r["eta"] == 0.0
    scale2 = max(np.max(np.abs(U[2])), np.max(np.abs(W[2])))
    assert r["mean_flow"] == pytest.approx(1e-9 / scale2, rel=1e-6)
    assert r["w00_alone"] == pytest.approx(1e-9 / np.max(np.abs(W[2])), rel=1e-6)
    lin = bench.rel_errors((got[0], got[1], None, None), (v, eta, None, None))
    assert set(lin) == {"v", "eta", "per_member"}


def test_config1_workload_is_the_16x33x16_couette_case():
    wl = bench.WORKLOADS["couette16"]
    g = wl["groups"][0]
    assert (g["mx"], g["my"], g["mz"], g["members"], g["re"], g["dt"]) == (16, 33, 16, 1, 400.0, 0.01)
    assert wl["noise"][0]["amp"] == 1e-2 and wl["noise"][0]["n_max"] == 2 and wl["noise"][0]["m_max"] == 2


def test_roofline_bound_follows_the_ridge_point():
    # ridge at 80 TFLOP/s over 6.8 TB/s: ~11.8 flop per byte
    assert bench.roofline_bound(7e8, 1e8, 80.0, 6800.0) == "hbm"
    assert bench.roofline_bound(3e9, 1e8, 80.0, 6800.0) == "alu"
    assert bench.roofline_bound(1e9, 0, 80.0, 6800.0) == "alu"
    # the fused stage of the headline (64x65x64, 4 members per launch) is below the ridge
    g = dict(bench.WORKLOADS["poiseuille64"]["groups"][0], members=4)
    w = bench.kernel_work("spec", g, "mixed")[1]
    b = bench.kernel_bytes("spec", g, "mixed")
    assert bench.roofline_bound(w, b, 80.5, 6799.3) == "hbm"
    # the plane stage is above it
    w = bench.kernel_work("plane", g, "mixed")[1]
    b = bench.kernel_bytes("plane", g, "mixed")
    assert bench.roofline_bound(w, b, 80.5, 6799.3) == "alu"


def test_parity_block_models_halve_the_operator_bytes_and_the_flops():
    """In parity blocks a matrix is its even and odd halves, Ny x 2 ceil(ceil(Ny/2)/2)
    floats (63 x 32 at Ny = 63 against 63 x 64 row-padded), and every product
    half the multiply-adds: the fused stage (fused_eo, fused_eo_ff), the
    step-by-step forcing and apply (simt_eo) and the y-derivatives (ygemm simt_eo)."""
    g = dict(bench.WORKLOADS["poiseuille64"]["groups"][0], members=4)
    S = 22 * 43 * 63 * 4
    nat = bench.kernel_bytes("spec", dict(g, _stage="fused_eo_ff"), "mixed")
    assert nat == pytest.approx(bench.kernel_bytes("spec", dict(g, _stage="fused_d2v"), "mixed")
                                - 483 * (10 / 3) * 63 * 32 * 4)
    h_nat = bench.kernel_bytes("helm", dict(g, _stage="simt"), "mixed")
    h_eo = bench.kernel_bytes("helm", dict(g, _stage="simt_eo"), "mixed")
    assert h_nat - h_eo == pytest.approx(484 * 2 * (5 / 3) * 63 * 32 * 4)
    for cls in ("forcing", "helm"):
        _, a, _ = bench.kernel_work(cls, dict(g, _stage="simt"), "mixed")
        _, b, _ = bench.kernel_work(cls, dict(g, _stage="simt_eo"), "mixed")
        assert b == pytest.approx(a / 2)
    assert bench.kernel_bytes("forcing", dict(g, _stage="simt_eo"), "mixed") == \
        bench.kernel_bytes("forcing", g, "mixed") == pytest.approx((40 + 16 * 4 / 3) * S)
    # the y-derivatives in parity blocks: half the flops, the same bytes
    _, a, _ = bench.kernel_work("yderiv", dict(g, _ygemm="simt"), "mixed")
    _, b, _ = bench.kernel_work("yderiv", dict(g, _ygemm="simt_eo"), "mixed")
    assert b == pytest.approx(a / 2) and a == pytest.approx(S * 3 * 2 * 2 * 63)
    assert bench.kernel_bytes("yderiv", dict(g, _ygemm="simt_eo"), "mixed") == bench.kernel_bytes("yderiv", g, "mixed")
