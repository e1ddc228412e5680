"""GPU path vs the CPU oracle, through the C ABI (needs a GPU)."""
import os

import numpy as np
import pytest

import dns_synth
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

FIELDS = ("v", "eta", "U", "W")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def group(flow, mx, my, mz, lx, lz, re, dt, members):
    return dict(flow=flow, mx=mx, my=my, mz=mz, lx=lx, lz=lz, re=re, dt=dt, members=members)


CFG1 = group("couette", 16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, 1)
CFG2 = group("poiseuille", 64, 65, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 8)


def _state(g, seed0, amp, **kw):
    return dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"],
                                seed0, amp, **kw)


def _oracle(g):
    return oracle.Channel(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["re"], g["dt"], g["flow"])


def _run(g, st, nsteps, precision="fp64", use_graph=False, ygemm="default", plane="default", helm="default"):
    ens = dns.Ensemble([g], precision=precision, use_graph=use_graph, ygemm=ygemm, plane=plane, helm=helm)
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.step(nsteps)
    out = ens.get_state(0)
    ens.close()
    return out


def test_config1_fp64_matches_oracle_after_100_steps():
    st = _state(CFG1, 1000, 1e-2, n_max=2, m_max=2)
    ref = _oracle(CFG1).step(tuple(st[k] for k in FIELDS), 100)
    got = _run(CFG1, st, 100)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-11, (name, rel(a, b))


@pytest.mark.parametrize("mx,my,mz,E", [(32, 49, 48, 3), (48, 21, 16, 5)])
def test_ragged_grids_fp64_match_oracle(mx, my, mz, E):
    g = group("couette", mx, my, mz, 1.75 * np.pi, 1.2 * np.pi, 500.0, 0.01, E)
    st = _state(g, 3000, 5e-2)
    ref = _oracle(g).step(tuple(st[k] for k in FIELDS), 5)
    got = _run(g, st, 5)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-12, (name, rel(a, b))


def test_config2_fp64_matches_oracle_few_steps():
    """Full size of the 64x65x64 Poiseuille ensemble (8 members), 3 steps."""
    st = _state(CFG2, 2000, 5e-2, n_max=4, m_max=4)
    ref = _oracle(CFG2).step(tuple(st[k] for k in FIELDS), 3)
    got = _run(CFG2, st, 3)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-12, (name, rel(a, b))


def test_config2_fp64_sampled_member_matches_oracle_over_100_steps():
    """Full-size 64x65x64 Poiseuille ensemble (8 members) advanced 100 steps by
    the FP64 path in the benchmark's launch configuration (CUDA graph, member
    blocks); the oracle follows one sampled member (members are independent: the
    GPU ran it inside the whole ensemble)."""
    st = _state(CFG2, 2000, 5e-2, n_max=4, m_max=4)
    ens = dns.Ensemble([CFG2], precision="fp64", use_graph=True)
    try:
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        ens.step(100)
        got = ens.get_state(0)
    finally:
        ens.close()
    e = 5
    ref = _oracle(CFG2).step(tuple(st[k][e:e + 1] for k in FIELDS), 100)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a[e:e + 1], b) < 1e-11, (name, rel(a[e:e + 1], b))


def _golden_channel128():
    path = os.path.join(os.path.dirname(__file__), "golden", "channel128_member5_2steps.txt")
    samples, prof, scale = {"v": [], "eta": []}, {"U": {}, "W": {}}, None
    with open(path) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "scale":
                scale = {"v": float(t[1]), "eta": float(t[2])}
            elif t[0] in samples:
                samples[t[0]].append((int(t[1]), int(t[2]), int(t[3]), complex(float(t[4]), float(t[5]))))
            else:
                prof[t[0]][int(t[1])] = float(t[2])
    return samples, prof, scale


def test_config5_fp64_sampled_member_matches_stored_oracle_values():
    """Full-size 128x97x128 constant-flux Poiseuille ensemble (Re_tau ~ 180, 16
    members, k^-5/3 noise at 10 %) advanced two steps by the FP64 path in the
    benchmark's launch configuration (CUDA graph, four member blocks, the
    cluster plane kernel); member 5 against 400 sampled v and eta values and
    the whole U, W profiles that the oracle wrote for it
    (tests/golden/make_channel128_samples.py, which calls only the oracle)."""
    lx, lz = 4 * np.pi, 4 * np.pi / 3
    g = group("poiseuille", 128, 97, 128, lx, lz, 3250.0, 0.002, 16)
    st = dns_synth.make_state(128, 97, 128, lx, lz, "poiseuille", 16, 5000, 1e-1, spectrum="kolmogorov")
    ens = dns.Ensemble([g], precision="fp64", use_graph=True)
    try:
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        ens.step(2)
        v, eta, U, W = ens.get_state(0, member0=5, count=1)
    finally:
        ens.close()
    samples, prof, scale = _golden_channel128()
    for name, a in (("v", v), ("eta", eta)):
        assert len(samples[name]) == 400
        err = max(abs(a[0, y, m, n] - c) for y, m, n, c in samples[name])
        assert err < 1e-11 * scale[name], (name, err / scale[name])
    for name, a in (("U", U), ("W", W)):
        ref = np.array([prof[name][j] for j in range(97)])
        assert np.abs(a[0] - ref).max() < 1e-11 * np.abs(ref).max(), name


@pytest.mark.parametrize("flow,mx,mz", [("couette", 16, 16), ("poiseuille", 32, 16)])
def test_maximum_wall_normal_resolution_matches_oracle(flow, mx, mz):
    """My = 129, the largest Chebyshev grid a group accepts (operators 127 x 127;
    the tensor-core kernels stop at 66, so the mixed path runs the register-
    tiled ones): FP64 vs the oracle, mixed vs FP64."""
    g = group(flow, mx, 129, mz, 2 * np.pi, np.pi, 1000.0, 0.002, 2)
    st = _state(g, 77, 2e-2)
    ref = _oracle(g).step(tuple(st[k] for k in FIELDS), 2)
    got = _run(g, st, 2)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-11, (name, rel(a, b))
    err = mixed_errors(_run(g, st, 2, "mixed"), got)
    assert np.all(err[:, :3] < 1e-6), err


@pytest.mark.parametrize("flow,my", [("couette", 5), ("poiseuille", 5), ("poiseuille", 7)])
def test_minimum_wall_normal_resolution_matches_oracle(flow, my):
    """My = 5 (three interior nodes, the smallest grid a group accepts) and 7:
    FP64 vs the oracle, then every y-contraction / implicit-apply pair of the
    mixed path (tensor-core tiles padded far beyond Ny) vs FP64."""
    g = group(flow, 32, my, 16, 2 * np.pi, np.pi, 500.0, 0.01, 3)
    st = _state(g, 91, 2e-2)
    ref = _oracle(g).step(tuple(st[k] for k in FIELDS), 3)
    got = _run(g, st, 3)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-11, (name, rel(a, b))
    for ygemm in ("simt", "tc"):
        for helm in ("simt", "tc"):
            err = mixed_errors(_run(g, st, 3, "mixed", ygemm=ygemm, helm=helm), got)
            assert np.all(err[:, :3] < 1e-6), (ygemm, helm, err)


def mixed_errors(mixed, ref):
    """Relative errors of the mixed step against the FP64 step, per member:
    v and eta each against their own maximum; the mean flow (U00, W00) as one
    velocity field against its maximum.  W00 alone is also reported: it is
    driven only by the plane mean <wv>, a strongly cancelling average of
    single-precision velocities, so its own-scale error sits near 1e-6."""
    out = []
    for e in range(ref[0].shape[0]):
        ev = rel(mixed[0][e], ref[0][e])
        ee = rel(mixed[1][e], ref[1][e])
        dm = max(np.abs(mixed[2][e] - ref[2][e]).max(), np.abs(mixed[3][e] - ref[3][e]).max())
        em = dm / max(np.abs(ref[2][e]).max(), np.abs(ref[3][e]).max())
        ew = rel(mixed[3][e], ref[3][e]) if np.abs(ref[3][e]).max() > 0 else 0.0
        out.append((ev, ee, em, ew))
    return np.array(out)


@pytest.mark.parametrize("ygemm,plane,helm", [("simt", "cta", "simt"), ("tc", "cta", "simt"), ("tc", "lines", "simt"),
                                              ("tc", "lines", "tc")])
def test_mixed_matches_fp64_over_50_steps(ygemm, plane, helm):
    g = group("couette", 32, 49, 32, 1.75 * np.pi, 1.2 * np.pi, 500.0, 0.01, 8)
    st = _state(g, 3000, 5e-2, n_max=4, m_max=4)
    a = _run(g, st, 50, "fp64")
    b = _run(g, st, 50, "mixed", ygemm=ygemm, plane=plane, helm=helm)
    err = mixed_errors(b, a)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 1e-5), err


def test_graph_replay_is_bitwise_equal_to_eager():
    g = group("poiseuille", 32, 33, 32, 2 * np.pi, np.pi, 1650.0, 0.005, 4)
    st = _state(g, 77, 5e-2)
    pin = dict(ygemm="tc", plane="lines", helm="tc")      # separate handles: no autotuner choice in between
    for prec in ("fp64", "mixed"):
        a = _run(g, st, 4, prec, use_graph=False, **pin)
        b = _run(g, st, 4, prec, use_graph=True, **pin)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,pin", [("fp64", {}),
                                           ("mixed", dict(ygemm="tc", plane="lines", helm="tc")),
                                           ("mixed", dict(ygemm="simt", plane="cta", helm="simt"))])
def test_member_alone_equals_member_in_batch(precision, pin):
    g = group("couette", 32, 33, 32, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, 6)
    st = _state(g, 500, 5e-2)
    full = _run(g, st, 3, precision, **pin)
    g1 = dict(g, members=1)
    one = {k: st[k][4:5] for k in FIELDS}
    alone = _run(g1, one, 3, precision, **pin)
    for a, b in zip(full, alone):
        assert np.array_equal(a[4:5], b)


def test_resume_is_bitwise(tmp_path):
    """Three steps, a checkpoint file (save_states / load_states), three more
    steps from it in a new handle: bitwise the six uninterrupted steps."""
    g = group("poiseuille", 16, 33, 16, 2 * np.pi, np.pi, 1650.0, 0.005, 2)
    st = _state(g, 9, 5e-2)
    direct = _run(g, st, 6)
    mid = _run(g, st, 3)
    path = str(tmp_path / "mid.npz")
    dns.save_states(path, [g], [mid])
    groups, states = dns.load_states(path)
    assert dns.same_groups(groups, [g])
    st2 = dict(zip(FIELDS, states[0]))
    resumed = _run(g, st2, 3)
    for a, b in zip(direct, resumed):
        assert np.array_equal(a, b)


def test_stats_match_oracle():
    g = group("poiseuille", 32, 33, 32, 2 * np.pi, np.pi, 1650.0, 0.005, 3)
    st = _state(g, 41, 5e-2)
    ch = _oracle(g)
    ref_state = ch.step(tuple(st[k] for k in FIELDS), 2)
    ref = ch.stats(ref_state)
    ens = dns.Ensemble([g], precision="fp64")
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.step(2)
    s = ens.stats(0)
    ens.close()
    for k in ("e_total", "e_pert", "tau_bottom", "tau_top", "bulk_flux"):
        assert np.abs(s[k] - ref[k]).max() <= 1e-12 * max(1.0, np.abs(ref[k]).max()), k
    # gamma = (Q - flux0) / flux1 cancels in Q - flux0, so it carries an absolute
    # error of about eps * Q / flux1 = 2.2e-16 * 1.33 / (dt * 1.33) ~ 5e-14
    assert np.abs(s["gamma"] - ch.last_gamma).max() < 1e-12
    assert np.all(s["max_div"] < 1e-13)
    for k in ("uu", "vv", "ww", "uv"):
        assert rel(s[k], ref[k]) < 1e-12, k
    assert np.all(s["nonfinite"] == 0)
    # the CFL number's velocity is synthesised in single precision
    assert np.allclose(s["cfl"], ref["cfl"], rtol=1e-5, atol=0), (s["cfl"], ref["cfl"])


@pytest.mark.parametrize("flow,mx,my,mz,precision,E", [("couette", 16, 33, 16, "fp64", 3),
                                                       ("poiseuille", 48, 21, 16, "mixed", 3),
                                                       ("poiseuille", 128, 33, 128, "mixed", 3),
                                                       ("couette", 64, 65, 64, "mixed", 8)])
def test_cfl_matches_oracle(flow, mx, my, mz, precision, E):
    """CFL number of every member (dt max of |u|/dx + |v|/dy + |w|/dz over the
    interior collocation points) against the oracle on ragged and 128-point
    grids and across two member blocks; the ensemble entry is the largest
    member's."""
    g = group(flow, mx, my, mz, 2 * np.pi, np.pi, 1000.0, 0.004, E)
    st = _state(g, 17, 1e-1)
    ens = dns.Ensemble([g], precision=precision)
    try:
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        s = ens.stats(0)
        rc, per, mean = dns.dns_stats(ens.h, 0, E, 0)
    finally:
        ens.close()
    ref = _oracle(g).stats(tuple(st[k] for k in FIELDS))["cfl"]
    assert np.allclose(s["cfl"], ref, rtol=1e-5, atol=0), (s["cfl"], ref)
    assert mean.cfl == max(s["cfl"])


def test_nonfinite_member_is_flagged_without_touching_others():
    g = group("couette", 16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, 3)
    st = _state(g, 5, 1e-2)
    st["v"][1, 3, 2, 1] = np.nan
    ens = dns.Ensemble([g], precision="fp64")
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.step(2)
    s = ens.stats(0)
    got = ens.get_state(0)
    ens.close()
    assert s["rc"] == dns.DNS_ERR_NONFINITE
    assert list(s["nonfinite"]) == [0, 1, 0]
    clean = {k: st[k][[0, 2]] for k in FIELDS}
    ref = _oracle(dict(g, members=2)).step(tuple(clean[k] for k in FIELDS), 2)
    for a, b in zip(got, ref):
        assert rel(a[[0, 2]], b) < 1e-12


def test_laminar_states_stay_steady_on_gpu():
    for flow in ("couette", "poiseuille"):
        g = group(flow, 32, 33, 32, 2 * np.pi, np.pi, 1650.0, 0.005, 2)
        st = _state(g, 0, 0.0)
        got = _run(g, st, 20)
        assert np.abs(got[2] - st["U"]).max() < 1e-13
        assert np.abs(got[0]).max() == 0.0


@pytest.mark.parametrize("plane", ["cta", "lines"])
@pytest.mark.parametrize("mx,mz", [(a, b) for a in (16, 32, 48, 64) for b in (16, 32, 48, 64)])
def test_mixed_matches_fp64_for_every_plane_shape(mx, mz, plane):
    g = group("poiseuille", mx, 33, mz, 2 * np.pi, np.pi, 1650.0, 0.005, 3)
    st = _state(g, 31, 5e-2)
    a = _run(g, st, 10, "fp64")
    b = _run(g, st, 10, "mixed", plane=plane)
    err = mixed_errors(b, a)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 1e-5), err


def test_bounded_device_wait_reports_timeout_and_context_survives():
    g = group("couette", 16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, 1)
    st = _state(g, 1000, 1e-2, n_max=2, m_max=2)
    pin = dict(ygemm="tc", plane="lines", helm="tc")      # two handles: no autotuner choice in between
    ens = dns.Ensemble([g], precision="mixed", **pin)
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    assert dns.dns_selftest_timeout(ens.h) == dns.DNS_ERR_TIMEOUT
    assert "gave up" in dns.dns_last_error(ens.h)
    ens.step(2)                      # the context is still usable
    got = ens.get_state(0)
    ens.close()
    ref = _run(g, st, 2, "mixed", **pin)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mx,my,mz,E", [(64, 65, 64, 8), (32, 33, 32, 5), (16, 21, 48, 64), (32, 49, 16, 1)])
def test_tensor_core_y_derivatives_match_fp64(mx, my, mz, E):
    """tcgen05 split-BF16 y-contraction and the register-tiled FP32 one, each
    against the FP64 step: both inside the 1e-6 budget (ragged grids, 1 to 64
    members)."""
    g = group("poiseuille", mx, my, mz, 2 * np.pi, np.pi, 1650.0, 0.005, E)
    st = _state(g, 71, 5e-2)
    ref = _run(g, st, 5, "fp64")
    for ygemm in ("simt", "tc"):
        err = mixed_errors(_run(g, st, 5, "mixed", ygemm=ygemm), ref)
        assert np.all(err[:, :3] < 1e-6), (ygemm, err)


def test_autotuner_picks_a_variant_caches_it_and_matches_that_variant(tmp_path):
    """The autotuned choices of a 32x32 mixed group (plane-stage kernel,
    y-contraction, per-wavenumber stage: the step-by-step apply variants after
    their y-derivatives and forcing, or the fused stage) are timed once,
    written to the cache, read back without new timing, and the step is
    bit-identical to requesting those variants."""
    g = group("poiseuille", 32, 33, 32, 2 * np.pi, np.pi, 1650.0, 0.005, 8)
    st = _state(g, 5, 5e-2)
    cache = str(tmp_path / "tune.txt")
    ens = dns.Ensemble([g], precision="mixed", autotune_cache=cache)
    choice = dns.dns_kernel_choice(ens.h, 0)
    plane = dns.dns_kernel_choice(ens.h, 0, "plane")
    helm = dns.dns_kernel_choice(ens.h, 0, "helm")
    assert choice in ("simt", "tc", "simt_eo") and plane in ("cta", "lines") and helm in ("simt", "tc", "fused", "fused_d2v",
                                                                                 "fused_eo", "fused_eo_ff", "simt_eo")
    assert helm not in ("fused", "fused_d2v", "fused_eo", "fused_eo_ff") or choice == "simt"
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.step(3)
    got = ens.get_state(0)
    ens.close()
    lines = sorted(ln for ln in open(cache) if ln.strip())
    keys = [ln.split()[0] for ln in lines]
    # keyed by the member block's size: 8 members run as 2 blocks of 4, tuned once;
    # the tile shapes: the fused stage's members per CTA, the y-derivative tile
    assert all(ln.split()[1:5] == ["32", "33", "32", "4"] for ln in lines)
    want = {"helm", "plane", "ygemm"} | ({"ytile"} if choice in ("simt", "simt_eo") else set()) | \
        ({"spec_ec"} if helm in ("fused", "fused_d2v", "fused_eo", "fused_eo_ff") else set()) | \
        ({"spec_cta"} if helm in ("fused_eo", "fused_eo_ff") else set())
    assert sorted(keys) == sorted(want)
    ens2 = dns.Ensemble([g], precision="mixed", autotune_cache=cache)   # read back, no new timing
    assert dns.dns_kernel_choice(ens2.h, 0) == choice
    assert dns.dns_kernel_choice(ens2.h, 0, "plane") == plane
    assert dns.dns_kernel_choice(ens2.h, 0, "helm") == helm
    ens2.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens2.step(3)
    again = ens2.get_state(0)                  # the cached choices reproduce the tuned run
    ens2.close()
    assert len([ln for ln in open(cache) if ln.strip()]) == len(lines)
    for a, b in zip(got, again):
        assert np.array_equal(a, b)
    ref = _run(g, st, 3, "mixed", ygemm=choice, plane=plane, helm=helm)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mx,my,mz,E", [(32, 49, 32, 8), (16, 33, 16, 3), (32, 33, 32, 64), (48, 65, 48, 5),
                                        (64, 65, 64, 2), (16, 21, 32, 33)])
def test_tensor_core_implicit_apply_matches_fp64(mx, my, mz, E):
    """tcgen05 implicit apply (split-BF16 operators and right-hand sides, FP32
    accumulation, one FP64 add): odd and large member counts (column padding,
    two column passes), the single-mode kx column pairs (m = 0), short and full
    operator heights."""
    g = group("poiseuille", mx, my, mz, 2 * np.pi, np.pi, 1650.0, 0.005, E)
    st = _state(g, 71, 5e-2)
    ref = _run(g, st, 10, "fp64")
    ens = dns.Ensemble([g], precision="mixed", helm="tc")
    assert dns.dns_kernel_choice(ens.h, 0, "helm") == "tc"
    ens.close()
    err = mixed_errors(_run(g, st, 10, "mixed", helm="tc"), ref)
    assert np.all(err[:, :3] < 1e-6), err


@pytest.mark.parametrize("mx,my,mz,E", [(32, 49, 32, 8), (16, 33, 16, 3), (32, 33, 32, 64), (64, 65, 64, 2),
                                        (16, 21, 32, 33), (128, 33, 128, 2)])
def test_persistent_implicit_apply_is_bitwise_the_one_shot_kernel(mx, my, mz, E):
    """The persistent, double-buffered implicit apply runs the same per-pair
    arithmetic as the one-CTA-per-pair kernel: identical results, bit for bit
    (member blocks, 128-point grids, odd member counts)."""
    g = group("poiseuille", mx, my, mz, 2 * np.pi, np.pi, 1650.0, 0.005, E)
    st = _state(g, 72, 5e-2)
    # separate handles: pin every autotuned variant (the cluster plane kernel is
    # the only one at 128 points)
    pin = dict(ygemm="simt", plane="cluster" if max(mx, mz) == 128 else "lines")
    ens = dns.Ensemble([g], precision="mixed", helm="persist", **pin)
    assert dns.dns_kernel_choice(ens.h, 0, "helm") == "persist"
    ens.close()
    a = _run(g, st, 4, "mixed", helm="persist", **pin)
    b = _run(g, st, 4, "mixed", helm="simt", **pin)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("mx,mz", [(128, 128), (128, 64), (64, 128)])
def test_fp64_cluster_plane_kernel_matches_oracle_on_128_grids(mx, mz):
    g = group("couette", mx, 25, mz, 1.75 * np.pi, 1.2 * np.pi, 500.0, 0.01, 2)
    st = _state(g, 4000, 5e-2, n_max=6, m_max=6)
    ref = _oracle(g).step(tuple(st[k] for k in FIELDS), 2)
    got = _run(g, st, 2)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-12, (name, rel(a, b))


@pytest.mark.parametrize("plane", ["cta", "cluster", "lines"])
def test_every_64x64_plane_kernel_matches_fp64(plane):
    g = group("poiseuille", 64, 33, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 3)
    st = _state(g, 17, 5e-2)
    ref = _run(g, st, 5, "fp64")
    err = mixed_errors(_run(g, st, 5, "mixed", plane=plane), ref)
    assert np.all(err[:, :3] < 1e-6), err


def test_channel_128x97x128_mixed_matches_fp64_over_50_steps():
    """Re_tau ~ 180 Poiseuille ensemble at full size (16 members, k^-5/3 noise,
    four member blocks), in the benchmark's launch configuration (CUDA graph,
    autotuned kernels), mixed against FP64 over the 50-step horizon."""
    g = group("poiseuille", 128, 97, 128, 4 * np.pi, 4 * np.pi / 3, 3250.0, 0.002, 16)
    st = dns_synth.make_state(128, 97, 128, g["lx"], g["lz"], "poiseuille", 16, 5000, 1e-1, spectrum="kolmogorov")
    ref = _run(g, st, 50, "fp64", use_graph=True)
    err = mixed_errors(_run(g, st, 50, "mixed", use_graph=True), ref)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 1e-5), err


@pytest.mark.parametrize("pin", [{}, dict(ygemm="simt", plane="lines", helm="simt"),
                                 dict(ygemm="simt", plane="lines", helm="tc")])
def test_headline_64x65x64_mixed_matches_fp64_over_50_steps_in_the_benchmark_launch(pin):
    """The benchmarked configuration itself: Poiseuille 64x65x64, 8 members (two
    member blocks of 4, concurrent graph branches), Re = 1650, dt = 0.005, 5 %
    noise, CUDA-graph replay, with the default kernels ({}: the fused stage) and
    with the step-by-step stage pinned; mixed against FP64 after 50 steps, per
    field and member.  (The tensor-core y-derivatives, FP32-accumulated, miss
    this budget here: eta 2.2e-6 after 50 steps.)"""
    st = _state(CFG2, 2000, 5e-2, n_max=4, m_max=4)
    ref = _run(CFG2, st, 50, "fp64", use_graph=True)
    err = mixed_errors(_run(CFG2, st, 50, "mixed", use_graph=True, **pin), ref)
    assert err.shape[0] == 8
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 3e-5), err


def test_config3_long_run_ensemble_statistics_mixed_match_fp64():
    """Couette Re = 500 minimal box, 32x49x32, 64 members, dt = 0.01, at full size
    over 1000 steps (the configuration's run length) in the launch configuration
    the benchmark times (CUDA graph, autotuned kernels, member blocks): the
    ensemble-mean profiles U(y), <u'u'>, <v'v'>, <w'w'>, <u'v'> of the mixed path
    within 1e-3 of the FP64 ones (relative to each profile's maximum), and every
    member's state within 1e-5 (measured: 8e-7 and 1.3e-6)."""
    g = group("couette", 32, 49, 32, 1.75 * np.pi, 1.2 * np.pi, 500.0, 0.01, 64)
    st = dns_synth.make_state(32, 49, 32, g["lx"], g["lz"], "couette", 64, 3000, 5e-2, n_max=4, m_max=4)
    out = {}
    for prec in ("fp64", "mixed"):
        ens = dns.Ensemble([g], precision=prec, use_graph=True)
        try:
            ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
            ens.step(1000)
            out[prec] = (ens.stats(0), ens.get_state(0))
        finally:
            ens.close()
    for k in ("U", "uu", "vv", "ww", "uv"):
        a, b = out["mixed"][0][k].mean(0), out["fp64"][0][k].mean(0)
        assert np.abs(a - b).max() < 1e-3 * np.abs(b).max(), k
    # per member: v, eta against their own maxima, the mean flow as one velocity field
    err = mixed_errors(out["mixed"][1], out["fp64"][1])
    assert np.all(err[:, :3] < 1e-5), err[:, :3].max(axis=0)


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_batch_groups_match_each_group_run_alone(precision, use_graph):
    """Three grids / Reynolds numbers / flows in one handle (the groups run as
    concurrent branches, captured in one graph or launched eagerly): each
    group's trajectory is bit-identical to the same group run on its own."""
    gs = [group("couette", 32, 33, 32, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.005, 3),
          group("couette", 48, 49, 48, 1.75 * np.pi, 1.2 * np.pi, 800.0, 0.005, 2),
          group("poiseuille", 64, 65, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 2)]
    sts = [_state(g, 4000 + 100 * i, np.linspace(1e-2, 5e-2, g["members"])) for i, g in enumerate(gs)]
    ens = dns.Ensemble(gs, precision=precision, use_graph=use_graph, ygemm="simt", plane="cta", helm="tc")
    for i, st in enumerate(sts):
        ens.set_state(i, st["v"], st["eta"], st["U"], st["W"])
    ens.step(3)
    together = [ens.get_state(i) for i in range(len(gs))]
    ens.close()
    for g, st, tog in zip(gs, sts, together):
        alone = _run(g, st, 3, precision, use_graph=True, ygemm="simt", plane="cta", helm="tc")
        for a, b in zip(tog, alone):
            assert np.array_equal(a, b)


def test_uneven_batch_at_full_size_sampled_members_match_oracle():
    """The 128-member uneven batch at full size in the benchmark's configuration
    (64 x Couette 32x33x32 Re 400, 32 x Couette 48x49x48 Re 800, 32 x Poiseuille
    64x65x64 Re 1650; amplitudes ramped 1e-2 to 5e-2; mixed precision, one CUDA
    graph, autotuned kernels, member blocks), 5 steps: one sampled member of each
    group against the oracle within the mixed path's 1e-6."""
    import bench
    wl = bench.WORKLOADS["uneven"]
    gs = [dict(g) for g in wl["groups"]]
    sts = [bench.initial_state(g, 0, nz) for g, nz in zip(gs, wl["noise"])]
    ens = dns.Ensemble(gs, precision="mixed", use_graph=True)
    picks = (37, 11, 29)
    try:
        for gi, st in enumerate(sts):
            ens.set_state(gi, st["v"], st["eta"], st["U"], st["W"])
        ens.step(5)
        got = [ens.get_state(gi, member0=e, count=1) for gi, e in enumerate(picks)]
    finally:
        ens.close()
    for gi, (g, st, e) in enumerate(zip(gs, sts, picks)):
        ref = _oracle(g).step(tuple(st[k][e:e + 1] for k in FIELDS), 5)
        err = mixed_errors(got[gi], ref)
        assert np.all(err[:, :3] < 1e-6), (gi, err)


def _shared_kx0(st):
    out = {k: np.array(st[k]) for k in FIELDS}
    for k in ("v", "eta"):
        out[k][:, :, :, 0] = out[k][:, :, :, 0].mean(axis=0)[None]
    for k in ("U", "W"):
        out[k][:] = out[k].mean(axis=0)[None]
    return out


@pytest.mark.parametrize("mx,my,mz,E", [(16, 33, 16, 3), (32, 49, 32, 5)])
def test_shared_mean_ensemble_fp64_matches_oracle(mx, my, mz, E):
    """S3T-type ensemble (members share the kx = 0 flow, driven by the
    member-averaged kx = 0 nonlinear terms and plane means): FP64 GPU vs the
    oracle's shared-mean mode, and the kx = 0 flow stays bit-identical across
    members on the GPU."""
    g = dict(group("couette", mx, my, mz, 2 * np.pi, 1.2 * np.pi, 1000.0, 0.01, E), shared_mean=True)
    st = _shared_kx0(_state(g, 600, 5e-2))
    ch = oracle.Channel(mx, my, mz, g["lx"], g["lz"], g["re"], g["dt"], "couette", shared_mean=True)
    ref = ch.step(tuple(st[k] for k in FIELDS), 4)
    got = _run(g, st, 4)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-12, (name, rel(a, b))
    for a in got[:2]:
        for e in range(1, E):
            assert np.array_equal(a[e, :, :, 0], a[0, :, :, 0])
    for a in got[2:]:
        for e in range(1, E):
            assert np.array_equal(a[e], a[0])
    plain = _run(dict(g, shared_mean=False), st, 4)
    assert rel(got[0], plain[0]) > 1e-9           # the coupling changes the trajectory


def test_shared_mean_ensemble_mixed_matches_fp64():
    g = dict(group("couette", 32, 49, 32, 2 * np.pi, 1.2 * np.pi, 1000.0, 0.01, 5), shared_mean=True)
    st = _shared_kx0(_state(g, 610, 5e-2))
    ref = _run(g, st, 20, "fp64")
    pin = dict(ygemm="tc", plane="lines", helm="simt")
    got = _run(g, st, 20, "mixed", **pin)
    err = mixed_errors(got, ref)
    assert np.all(err[:, :3] < 1e-6), err
    for a in got[:2]:
        for e in range(1, 5):
            assert np.array_equal(a[e, :, :, 0], a[0, :, :, 0])


def test_shared_mean_with_one_member_is_the_plain_step():
    g = group("couette", 16, 33, 16, 2 * np.pi, 1.2 * np.pi, 1000.0, 0.01, 1)
    st = _state(g, 620, 5e-2)
    for prec in ("fp64", "mixed"):
        pin = {} if prec == "fp64" else dict(ygemm="tc", plane="lines", helm="tc")
        a = _run(dict(g, shared_mean=True), st, 3, prec, **pin)
        b = _run(g, st, 3, prec, **pin)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("block", [0, 20, 3])
def test_member_blocks_are_invisible_to_the_caller(block):
    """A group of 40 members runs internally as concurrent member blocks
    (automatic: 4 x 10; 2 x 20; 13 blocks of 3 or 4).  Members straddling a
    block boundary evolve bit for bit as in a single-block group of 8, partial
    set/get across the boundary round-trips, and the statistics match the small
    group's member by member."""
    g = dict(group("couette", 16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01, 40), member_block=block)
    st = _state(g, 900, 5e-2)
    sub = {k: st[k][16:24] for k in FIELDS}
    g8 = dict(g, members=8, member_block=8)
    for prec, pin in (("fp64", {}), ("mixed", dict(ygemm="tc", plane="lines", helm="simt"))):
        full = _run(g, st, 2, prec, use_graph=True, **pin)
        ref = _run(g8, sub, 2, prec, use_graph=True, **pin)
        for a, b in zip(full, ref):
            assert np.array_equal(a[16:24], b)
    ens = dns.Ensemble([g], precision="fp64")
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.set_state(0, *(sub[k][::-1].copy() for k in FIELDS), member0=16)      # overwrite across the boundary
    got = ens.get_state(0, member0=14, count=12)
    assert np.array_equal(got[0][2:10], sub["v"][::-1]) and np.array_equal(got[0][:2], st["v"][14:16])
    assert np.array_equal(got[2][10:], st["U"][24:26])
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    ens.step(1)
    s40 = ens.stats(0)
    ens.close()
    e8 = dns.Ensemble([g8], precision="fp64")
    e8.set_state(0, *(sub[k] for k in FIELDS))
    e8.step(1)
    s8 = e8.stats(0)
    e8.close()
    for k in ("e_total", "e_pert", "tau_bottom", "max_div"):
        assert np.array_equal(s40[k][16:24], s8[k]), k
    assert np.array_equal(s40["uu"][16:24], s8["uu"])


@pytest.mark.parametrize("mx,my,mz,E", [(16, 33, 16, 2), (32, 49, 32, 3), (64, 33, 48, 2)])
def test_rotational_form_fp64_matches_oracle(mx, my, mz, E):
    g = dict(group("poiseuille", mx, my, mz, 2 * np.pi, np.pi, 1650.0, 0.005, E), form="rotational")
    st = _state(g, 700, 5e-2)
    ch = oracle.Channel(mx, my, mz, g["lx"], g["lz"], g["re"], g["dt"], "poiseuille", form="rotational")
    ref = ch.step(tuple(st[k] for k in FIELDS), 4)
    got = _run(g, st, 4)
    for a, b, name in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-12, (name, rel(a, b))
    adv = _run(dict(g, form="advective"), st, 4)
    assert rel(got[0], adv[0]) > 1e-14         # a different discretisation of N


@pytest.mark.parametrize("mx,mz", [(16, 16), (32, 48), (48, 32), (64, 64), (64, 16)])
def test_rotational_form_mixed_matches_fp64(mx, mz):
    g = dict(group("poiseuille", mx, 33, mz, 2 * np.pi, np.pi, 1650.0, 0.005, 3), form="rotational")
    st = _state(g, 710, 5e-2)
    ref = _run(g, st, 10, "fp64")
    ens = dns.Ensemble([g], precision="mixed")
    assert dns.dns_kernel_choice(ens.h, 0, "plane") == "lines"
    ens.close()
    err = mixed_errors(_run(g, st, 10, "mixed"), ref)
    assert np.all(err[:, :3] < 1e-6), err


@pytest.mark.parametrize("flow,mx,my,mz,E,extra", [
    ("poiseuille", 32, 33, 32, 3, {}),
    ("couette", 48, 49, 48, 5, {}),
    ("poiseuille", 16, 21, 48, 20, dict(member_block=20)),      # one block of 20: member chunks 8, 8, 4
    ("couette", 64, 65, 64, 4, dict(form="rotational")),
    ("poiseuille", 32, 97, 16, 2, {}),
    ("couette", 16, 7, 16, 3, {}),
])
def test_fused_stage_matches_fp64_and_the_step_by_step_stage(flow, mx, my, mz, E, extra):
    """The fused per-wavenumber stage (forcing, RK combination, implicit apply,
    y-derivatives of the new state, mean flow with the last-CTA finish) against
    the FP64 step over 20 steps (1e-6 per field and member; the mean flow as one
    field), and against the step-by-step mixed stage (the same arithmetic up to
    summation order).  W00 on its own scale: O(1e-5) in size and driven only by
    the plane mean <wv>, an average of single-precision products that cancels
    strongly, so its own-scale error follows the single-precision inputs
    (measured up to 1.1e-5 here): held at 3e-5, and the fused stage within a
    factor 2 of the step-by-step one."""
    g = dict(group(flow, mx, my, mz, 2 * np.pi, np.pi, 1650.0 if flow == "poiseuille" else 400.0, 0.005, E), **extra)
    st = _state(g, 91, 5e-2)
    ref = _run(g, st, 20, "fp64")
    fused = _run(g, st, 20, "mixed", use_graph=True, helm="fused")
    chain = _run(g, st, 20, "mixed", helm="simt", ygemm="simt")
    err = mixed_errors(fused, ref)
    err_chain = mixed_errors(chain, ref)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 3e-5), err
    assert np.all(err[:, 3] <= 2.0 * err_chain[:, 3] + 1e-7), (err, err_chain)
    assert np.all(mixed_errors(fused, chain)[:, :3] < 1e-6)


def test_fused_stage_member_alone_equals_member_in_batch_and_resumes_bitwise():
    """A member alone = the same member in a batch (bitwise; the plane kernel
    pinned: separate handles are autotuned separately), and 3 + 3 steps through
    get/set (the new state's derivatives then come from the separate
    y-derivative kernel) = 6 steps within the mixed budget.  Not bitwise:
    setting a state replaces the n = 0 column by its Hermitian part, a change
    at the last bit of the FP64 state that can flip the rounding of a
    single-precision intermediate (1e-8 relative differences after 3 steps)."""
    g = group("poiseuille", 32, 33, 32, 2 * np.pi, np.pi, 1650.0, 0.005, 6)
    st = _state(g, 93, 5e-2)
    pin = dict(helm="fused", plane="lines")
    whole = _run(g, st, 6, "mixed", **pin)
    g1 = dict(g, members=1)
    one = _run(g1, {k: st[k][2:3] for k in FIELDS}, 6, "mixed", **pin)
    for a, b in zip(whole, one):
        assert np.array_equal(a[2:3], b)
    half = _run(g, st, 3, "mixed", **pin)
    again = _run(g, dict(zip(FIELDS, half)), 3, "mixed", **pin)
    err = mixed_errors(again, whole)
    assert np.all(err[:, :3] < 1e-6), err


@pytest.mark.parametrize("flow,mx,my,mz,E,extra", [
    ("poiseuille", 64, 65, 64, 8, {}),                        # the benchmarked case: two blocks of 4
    ("couette", 16, 21, 48, 3, {}),                           # Ny = 19: K padded to 32
    ("poiseuille", 32, 49, 32, 5, {}),                        # member chunks of 4 and 1
    ("couette", 48, 33, 48, 1, {}),
    ("poiseuille", 32, 33, 16, 6, dict(member_block=6)),      # chunks of 4 and 2
    ("couette", 64, 65, 64, 4, dict(form="rotational")),
])
def test_fused_d2v_is_bitwise_the_separate_digit_kernel(flow, mx, my, mz, E, extra):
    """The fused stage with the tensor-core D2 v inside it (digits of the new
    state, the MMAs and the TMEM read-back in the same launch) runs the digit
    arithmetic of the separate D2 v kernel: each level is an exact integer sum,
    so the state after 4 steps (CUDA graph) is bit for bit the one of the fused
    stage followed by the separate kernel."""
    g = dict(group(flow, mx, my, mz, 2 * np.pi, np.pi, 1650.0 if flow == "poiseuille" else 400.0, 0.005, E), **extra)
    st = _state(g, 97, 5e-2)
    ens = dns.Ensemble([g], precision="mixed", helm="fused_d2v", plane="lines")
    assert dns.dns_kernel_choice(ens.h, 0, "helm") == "fused_d2v"
    ens.close()
    sep = _run(g, st, 4, "mixed", use_graph=True, helm="fused", plane="lines")
    inside = _run(g, st, 4, "mixed", use_graph=True, helm="fused_d2v", plane="lines")
    for a, b, name in zip(sep, inside, FIELDS):
        assert np.array_equal(a, b), name


def test_fused_d2v_request_falls_back_where_it_cannot_run():
    """Above Ny = 64 the stage sums D2 v in float-float and has no digit image:
    a request for the fused D2 v runs the plain fused stage there."""
    g = group("poiseuille", 32, 97, 16, 2 * np.pi, np.pi, 1650.0, 0.005, 2)
    ens = dns.Ensemble([g], precision="mixed", helm="fused_d2v")
    try:
        assert dns.dns_kernel_choice(ens.h, 0, "helm") == "fused"
    finally:
        ens.close()


def test_fused_stage_shape_specialisations_are_bitwise_the_generic_kernel():
    """At Ny = 63 the fused stage has instantiations with the wall-normal size
    and the members per CTA as compile-time constants (4 and 2 here); three
    members run the generic kernel.  Members evolve independently, so the
    first members of the four- and two-member runs equal the three-member run's
    bit for bit after 3 steps."""
    g4 = group("poiseuille", 64, 65, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 4)
    st = _state(g4, 99, 5e-2)
    pin = dict(helm="fused", plane="lines")
    four = _run(g4, st, 3, "mixed", **pin)
    three = _run(dict(g4, members=3), {k: st[k][:3] for k in FIELDS}, 3, "mixed", **pin)
    two = _run(dict(g4, members=2), {k: st[k][:2] for k in FIELDS}, 3, "mixed", **pin)
    for a, b, c, name in zip(four, three, two, FIELDS):
        assert np.array_equal(a[:3], b), name
        assert np.array_equal(a[:2], c), name


@pytest.mark.parametrize("stage", ["fused_eo", "fused_eo_ff"])
@pytest.mark.parametrize("flow,mx,my,mz,E,extra", [
    ("poiseuille", 32, 33, 32, 3, {}),
    ("couette", 48, 49, 48, 5, {}),
    ("poiseuille", 16, 21, 48, 20, dict(member_block=20)),      # one block of 20: member chunks
    ("couette", 64, 65, 64, 4, dict(form="rotational")),
    ("couette", 16, 7, 16, 3, {}),                              # Ny = 5: parity parts of 3 and 2 rows
    ("poiseuille", 32, 34, 16, 2, {}),                          # even Ny: no centre row
    ("poiseuille", 32, 97, 16, 2, {}),                          # Ny = 95: float-float D2 v only
])
def test_fused_stage_in_parity_blocks_matches_fp64_and_the_natural_order_stage(stage, flow, mx, my, mz, E, extra):
    """The fused stage in parity blocks (every operator as its even and odd
    halves; D2 v from the digit kernel, or summed inside in float-float)
    against the FP64 step over 20 steps (1e-6 per field and member, W00 on its
    own scale at 3e-5) and against the fused stage in the natural order (the
    same arithmetic regrouped: within the budget).  Above Ny = 64 there is no
    digit kernel: only the float-float form runs."""
    g = dict(group(flow, mx, my, mz, 2 * np.pi, np.pi, 1650.0 if flow == "poiseuille" else 400.0, 0.005, E), **extra)
    st = _state(g, 91, 5e-2)
    ens = dns.Ensemble([g], precision="mixed", helm=stage)
    got = dns.dns_kernel_choice(ens.h, 0, "helm")
    ens.close()
    if stage == "fused_eo" and my - 2 > 64:
        assert got == "fused"
        return
    assert got == stage
    ref = _run(g, st, 20, "fp64")
    par = _run(g, st, 20, "mixed", use_graph=True, helm=stage)
    nat = _run(g, st, 20, "mixed", use_graph=True, helm="fused")
    err = mixed_errors(par, ref)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 3e-5), err
    assert np.all(mixed_errors(par, nat)[:, :3] < 1e-6)


@pytest.mark.parametrize("flow,mx,my,mz,E,extra", [
    ("couette", 32, 33, 32, 5, {}),
    ("poiseuille", 64, 65, 64, 4, {}),
    ("poiseuille", 16, 21, 48, 20, dict(member_block=20)),      # one block of 20: member chunks
    ("couette", 48, 49, 48, 3, dict(form="rotational")),
    ("couette", 16, 7, 16, 3, {}),                              # Ny = 5: parity parts of 3 and 2 rows
    ("poiseuille", 32, 34, 16, 2, {}),                          # even Ny: no centre row
    ("poiseuille", 32, 97, 16, 2, {}),                          # Ny = 95
])
def test_step_by_step_stage_in_parity_blocks_matches_fp64_and_the_natural_order_stage(flow, mx, my, mz, E, extra):
    """The step-by-step stage with its forcing (D1) and implicit apply (M - I,
    P) in parity blocks against the FP64 step over 20 steps (1e-6 per field and
    member, W00 on its own scale at 3e-5) and against the same stage in the
    natural order (the same products regrouped: within the budget)."""
    g = dict(group(flow, mx, my, mz, 2 * np.pi, np.pi, 1650.0 if flow == "poiseuille" else 400.0, 0.005, E), **extra)
    st = _state(g, 93, 5e-2)
    ens = dns.Ensemble([g], precision="mixed", helm="simt_eo")
    got = dns.dns_kernel_choice(ens.h, 0, "helm")
    ens.close()
    assert got == "simt_eo"
    ref = _run(g, st, 20, "fp64")
    par = _run(g, st, 20, "mixed", use_graph=True, helm="simt_eo")
    nat = _run(g, st, 20, "mixed", use_graph=True, helm="simt")
    err = mixed_errors(par, ref)
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 3e-5), err
    assert np.all(mixed_errors(par, nat)[:, :3] < 1e-6)


@pytest.mark.parametrize("flow,mx,my,mz,E,extra", [
    ("couette", 32, 49, 32, 6, {}),
    ("poiseuille", 16, 21, 48, 20, dict(member_block=20)),      # one block of 20
    ("couette", 48, 49, 48, 3, dict(form="rotational")),
    ("couette", 16, 7, 16, 3, {}),                              # Ny = 5
    ("poiseuille", 32, 34, 16, 2, {}),                          # even Ny: no centre row
    ("poiseuille", 32, 97, 16, 4, {}),                          # Ny = 95
])
def test_y_derivatives_in_parity_blocks_match_fp64_and_the_natural_order_kernel(flow, mx, my, mz, E, extra):
    """The register-tiled y-derivatives in parity blocks (D1 and D2 as their
    even and odd halves, D2 v in float-float from the float-float parts of the
    FP64 state), in the step-by-step stage with either apply, against the FP64
    step over 20 steps (1e-6 per field and member, W00 on its own scale at
    3e-5) and against the natural-order kernel (within the budget)."""
    g = dict(group(flow, mx, my, mz, 2 * np.pi, np.pi, 1650.0 if flow == "poiseuille" else 400.0, 0.005, E), **extra)
    st = _state(g, 95, 5e-2)
    ens = dns.Ensemble([g], precision="mixed", ygemm="simt_eo", helm="simt")
    assert dns.dns_kernel_choice(ens.h, 0, "ygemm") == "simt_eo"
    ens.close()
    ref = _run(g, st, 20, "fp64")
    nat = _run(g, st, 20, "mixed", use_graph=True, ygemm="simt", helm="simt")
    for helm in ("simt", "simt_eo"):
        par = _run(g, st, 20, "mixed", use_graph=True, ygemm="simt_eo", helm=helm)
        err = mixed_errors(par, ref)
        assert np.all(err[:, :3] < 1e-6), (helm, err)
        assert np.all(err[:, 3] < 3e-5), (helm, err)
        assert np.all(mixed_errors(par, nat)[:, :3] < 1e-6), helm


def test_step_by_step_stage_in_parity_blocks_keeps_members_independent():
    """Members evolve independently in the parity-block forcing and apply as
    anywhere else: the first members of a 5-member run (one block; the
    forcing's column tiles and the apply's CTAs hold other member counts) equal
    a 3-member run bit for bit after 3 steps, eager and graph replay alike."""
    g = group("couette", 32, 33, 32, 2 * np.pi, np.pi, 400.0, 0.005, 5)
    st = _state(g, 97, 5e-2)
    five = _run(dict(g, member_block=5), st, 3, "mixed", helm="simt_eo", plane="lines")
    three = _run(dict(g, members=3), {k: st[k][:3] for k in FIELDS}, 3, "mixed", use_graph=True, helm="simt_eo",
                 plane="lines")
    for a, b, name in zip(five, three, FIELDS):
        assert np.array_equal(a[:3], b), name


@pytest.mark.parametrize("stage", ["fused_eo", "fused_eo_ff"])
def test_headline_in_parity_blocks_matches_fp64_over_50_steps(stage):
    """The benchmarked configuration (64x65x64, 8 members in two blocks, graph)
    with the fused stage in parity blocks, mixed against FP64 after 50 steps."""
    st = _state(CFG2, 2000, 5e-2, n_max=4, m_max=4)
    ref = _run(CFG2, st, 50, "fp64", use_graph=True)
    err = mixed_errors(_run(CFG2, st, 50, "mixed", use_graph=True, helm=stage), ref)
    assert err.shape[0] == 8
    assert np.all(err[:, :3] < 1e-6), err
    assert np.all(err[:, 3] < 3e-5), err


def test_parity_block_stage_ctas_per_sm_do_not_change_the_result(tmp_path):
    """The register budget of the parity-block fused stage (2 or 3 CTAs per SM,
    a tuned shape read here from a cache file) changes no result: 3 steps of
    the headline grid are bitwise the same under both."""
    g = group("poiseuille", 64, 65, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 4)
    st = _state(g, 101, 5e-2)
    out = []
    for minb in (2, 3):
        cache = tmp_path / ("tune%d.txt" % minb)
        cache.write_text("spec_cta 64 65 64 4 %d\n" % minb)
        ens = dns.Ensemble([g], precision="mixed", helm="fused_eo", plane="lines", autotune_cache=str(cache))
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        ens.step(3)
        out.append(ens.get_state(0))
        ens.close()
    for a, b, name in zip(out[0], out[1], FIELDS):
        assert np.array_equal(a, b), name


@pytest.mark.parametrize("stage", ["fused_eo", "fused_eo_ff"])
def test_parity_block_stage_resumes_through_get_and_set(stage):
    """3 + 3 steps through get/set (the derivatives of the set state then come
    from the parity-block derivative kernel, as the stage computes them) = 6
    steps within the mixed budget, and a member alone = the same member in a
    batch, bitwise."""
    g = group("poiseuille", 64, 65, 64, 2 * np.pi, np.pi, 1650.0, 0.005, 4)
    st = _state(g, 103, 5e-2)
    pin = dict(helm=stage, plane="lines")
    whole = _run(g, st, 6, "mixed", **pin)
    half = _run(g, st, 3, "mixed", **pin)
    again = _run(g, dict(zip(FIELDS, half)), 3, "mixed", **pin)
    err = mixed_errors(again, whole)
    assert np.all(err[:, :3] < 1e-6), err
    one = _run(dict(g, members=1), {k: st[k][1:2] for k in FIELDS}, 6, "mixed", **pin)
    for a, b in zip(whole, one):
        assert np.array_equal(a[1:2], b)
