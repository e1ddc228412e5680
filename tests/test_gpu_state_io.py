"""State upload and download through the C ABI (dns_set_state / dns_get_state)
with every kind of buffer a caller may pass: pageable host memory (staged
copies), page-locked host memory (read and written by the pack and unpack
kernels over the CPU-GPU link), page-locked memory at an offset inside a larger
allocation, and device memory.  Every path must move the same bytes: the
states they give back are compared bitwise, over member ranges that cross the
boundary between two member blocks and with destinations left out."""
import numpy as np
import pytest

import dns_synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

G = dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=8,
         member_block=4)
# every handle in these comparisons runs the same kernel variants (the autotuner
# decides per handle, and near-equal timings may resolve differently)
PIN = dict(ygemm="tc", plane="lines", helm="simt")


def _pinned(a, offset=0):
    """A page-locked copy of array a (float64 view), optionally placed `offset`
    doubles into a larger page-locked allocation."""
    flat = np.ascontiguousarray(a).view(np.float64).ravel()
    big = torch.zeros(flat.size + offset + 3, dtype=torch.float64).pin_memory()
    t = big[offset:offset + flat.size]
    t.copy_(torch.from_numpy(flat))
    return big, t


def _device(a, offset=0):
    """The same on the device: kernels read it directly when aligned, staged
    device-to-device copies serve it otherwise."""
    flat = np.ascontiguousarray(a).view(np.float64).ravel()
    big = torch.zeros(flat.size + offset + 3, dtype=torch.float64, device="cuda")
    t = big[offset:offset + flat.size]
    t.copy_(torch.from_numpy(flat))
    return big, t


def _host(t, like):
    return t.numpy().view(like.dtype).reshape(like.shape)


def _ptr(t):
    return t.data_ptr() if t is not None else None


def _state():
    return dns_synth.make_state(G["mx"], G["my"], G["mz"], G["lx"], G["lz"], G["flow"], G["members"], 41, 5e-2)


@pytest.mark.parametrize("offset", [0, 2, 5])   # doubles: 5 leaves v, eta 8-byte aligned only (staged copies)
def test_pinned_and_device_buffers_move_the_same_state_as_pageable_ones(offset):
    st = _state()
    a = dns.Ensemble([G], precision="mixed", **PIN)
    b = dns.Ensemble([G], precision="mixed", **PIN)
    c = dns.Ensemble([G], precision="mixed", **PIN)
    try:
        a.set_state(0, st["v"], st["eta"], st["U"], st["W"])               # pageable numpy: staged copies
        keep = [_pinned(st[k], offset) for k in ("v", "eta", "U", "W")]   # page-locked: direct reads
        dns.dns_set_state(b.h, 0, 0, G["members"], *[_ptr(t) for _, t in keep], 0)
        dev = [_device(st[k], offset) for k in ("v", "eta", "U", "W")]
        dns.dns_set_state(c.h, 0, 0, G["members"], *[_ptr(t) for _, t in dev], 1)   # device pointers
        for ens in (a, b, c):
            ens.step(3)
        ref = a.get_state(0)
        for ens in (b, c):
            got = ens.get_state(0)
            for x, y in zip(got, ref):
                assert np.array_equal(x, y)
        # download into page-locked buffers (direct writes) and device buffers
        outs = [_pinned(np.zeros_like(r), offset) for r in ref]
        dns.dns_get_state(a.h, 0, 0, G["members"], *[_ptr(t) for _, t in outs], 0)
        for (_, t), r in zip(outs, ref):
            assert np.array_equal(_host(t, r), r)
        douts = [_device(np.zeros_like(r), offset) for r in ref]
        dns.dns_get_state(a.h, 0, 0, G["members"], *[_ptr(t) for _, t in douts], 1)
        for (_, t), r in zip(douts, ref):
            assert np.array_equal(t.cpu().numpy().view(r.dtype).reshape(r.shape), r)
    finally:
        for ens in (a, b, c):
            ens.close()


def test_partial_member_ranges_across_blocks_and_missing_destinations():
    st = _state()
    a = dns.Ensemble([G], precision="mixed", **PIN)
    b = dns.Ensemble([G], precision="mixed", **PIN)
    try:
        a.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        b.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        # members 3..6 (two in each block) replaced from page-locked buffers in b,
        # from pageable ones in a
        st2 = _state()
        sub = {k: np.ascontiguousarray(st2[k][3:7] * 0.5) for k in ("v", "eta", "U", "W")}
        a.set_state(0, sub["v"], sub["eta"], sub["U"], sub["W"], member0=3)
        keep = [_pinned(sub[k]) for k in ("v", "eta", "U", "W")]
        dns.dns_set_state(b.h, 0, 3, 4, *[_ptr(t) for _, t in keep], 0)
        a.step(2)
        b.step(2)
        ref = a.get_state(0)
        got = b.get_state(0)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
        # members 2..6 into page-locked buffers, eta and W left out
        r5 = [r[2:7] for r in ref]
        outs = [_pinned(np.zeros_like(r)) for r in r5]
        dns.dns_get_state(b.h, 0, 2, 5, _ptr(outs[0][1]), None, _ptr(outs[2][1]), None, 0)
        assert np.array_equal(_host(outs[0][1], r5[0]), r5[0])
        assert np.array_equal(_host(outs[2][1], r5[2]), r5[2])
        assert not _host(outs[1][1], r5[1]).any() and not _host(outs[3][1], r5[3]).any()
    finally:
        a.close()
        b.close()


def test_linear_group_state_through_page_locked_buffers():
    my, mz, lz = 33, 32, np.pi
    g = dict(flow="couette", mx=0, my=my, mz=mz, lx=2 * np.pi, lz=lz, re=1000.0, dt=0.02, members=3,
             linear=True, kx_index=1)
    b = dns_synth.make_base_flow(my, mz, lz, "couette", 5, streak=0.3, roll=0.03)
    d = dns_synth.make_disturbances(my, mz, lz, 3, 17)
    e1 = dns.Ensemble([g], precision="fp64")
    e2 = dns.Ensemble([g], precision="fp64")
    try:
        for e in (e1, e2):
            e.set_base_flow(0, b["U"], b["V"], b["W"])
        e1.set_state(0, d["v"][..., None], d["eta"][..., None])
        keep = [_pinned(np.ascontiguousarray(d[k][..., None])) for k in ("v", "eta")]
        dns.dns_set_state(e2.h, 0, 0, 3, _ptr(keep[0][1]), _ptr(keep[1][1]), None, None, 0)
        e1.step(3)
        e2.step(3)
        r1, r2 = e1.get_state(0), e2.get_state(0)
        assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
        outs = [_pinned(np.zeros_like(r1[i])) for i in (0, 1)]
        dns.dns_get_state(e2.h, 0, 0, 3, _ptr(outs[0][1]), _ptr(outs[1][1]), None, None, 0)
        assert np.array_equal(_host(outs[0][1], r1[0]), r1[0]) and np.array_equal(_host(outs[1][1], r1[1]), r1[1])
    finally:
        e1.close()
        e2.close()


G2 = dict(flow="couette", mx=16, my=25, mz=32, lx=2 * np.pi, lz=np.pi, re=800.0, dt=0.01, members=5,
          member_block=2)


def _states(groups, seed):
    return [dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"], seed + i,
                                 5e-2) for i, g in enumerate(groups)]


def _reference(groups, sts, nsteps, **kw):
    ens = dns.Ensemble(groups, precision="mixed", **PIN, **kw)
    try:
        for gi, st in enumerate(sts):
            ens.set_state(gi, st["v"], st["eta"], st["U"], st["W"])
        ens.step(nsteps)
        return [ens.get_state(gi) for gi in range(len(groups))]
    finally:
        ens.close()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("nsteps", [0, 1, 3, 17])   # 17: above the whole-call graph's limit
def test_advance_equals_set_step_get(use_graph, nsteps):
    """dns_advance over an uneven batch (a group of two member blocks of 4 and a
    group of 5 members in blocks of 3 and 2) = dns_set_state + dns_step + dns_get_state,
    bitwise, with pageable buffers and with page-locked ones."""
    groups = [G, G2]
    sts = _states(groups, 7)
    ref = _reference(groups, sts, nsteps, use_graph=use_graph)
    ens = dns.Ensemble(groups, precision="mixed", use_graph=use_graph, **PIN)
    try:
        got = ens.advance(nsteps, [(s["v"], s["eta"], s["U"], s["W"]) for s in sts])   # pageable
        for a, b in zip(got, ref):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
        # page-locked buffers, twice in a row (the second call replays the captured advance graph)
        keep_in = [[_pinned(s[k]) for k in ("v", "eta", "U", "W")] for s in sts]
        keep_out = [[_pinned(np.zeros_like(x)) for x in r] for r in ref]
        for _ in range(2):
            dns.dns_advance(ens.h, nsteps, [tuple(_ptr(t) for _, t in kin) for kin in keep_in],
                            [tuple(_ptr(t) for _, t in kout) for kout in keep_out], 0)
            for kout, r in zip(keep_out, ref):
                for (_, t), x in zip(kout, r):
                    assert np.array_equal(_host(t, x), x)
    finally:
        ens.close()


def test_advance_without_upload_or_download_continues_the_current_state():
    groups = [G, G2]
    sts = _states(groups, 11)
    ref = _reference(groups, sts, 4, use_graph=True)
    ens = dns.Ensemble(groups, precision="mixed", use_graph=True, **PIN)
    try:
        ens.advance(1, [(s["v"], s["eta"], s["U"], s["W"]) for s in sts])
        dns.dns_advance(ens.h, 2, None, None, 0)                         # keep the state, read nothing
        outs = [tuple(np.zeros_like(x) for x in r) for r in ref]
        dns.dns_advance(ens.h, 1, None, [(o[0].ctypes.data, None, o[2].ctypes.data, None) for o in outs], 0)
        for o, r in zip(outs, ref):
            assert np.array_equal(o[0], r[0]) and np.array_equal(o[2], r[2])
            assert not o[1].any() and not o[3].any()
        got = [ens.get_state(gi) for gi in range(2)]
        for a, b in zip(got, ref):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    finally:
        ens.close()


def test_advance_with_stochastic_forcing_and_a_linear_group():
    gf = dict(G, members=6, member_block=3)
    my, mz, lz = 33, 32, np.pi
    gl = dict(flow="couette", mx=0, my=my, mz=mz, lx=2 * np.pi, lz=lz, re=1000.0, dt=0.02, members=3,
              linear=True, kx_index=1)
    b = dns_synth.make_base_flow(my, mz, lz, "couette", 5, streak=0.3, roll=0.03)
    d = dns_synth.make_disturbances(my, mz, lz, 3, 17)
    st = _states([gf], 3)[0]
    out = []
    for mode in ("separate", "advance"):
        ens = dns.Ensemble([gf, gl], precision="mixed", use_graph=True, **PIN)
        try:
            ens.set_stochastic_forcing(0, 1, 4, 1e-3, 99)
            ens.set_base_flow(1, b["U"], b["V"], b["W"])
            if mode == "separate":
                ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
                ens.set_state(1, d["v"][..., None], d["eta"][..., None])
                ens.step(3)
                out.append([ens.get_state(0), ens.get_state(1)])
            else:
                out.append(ens.advance(3, [(st["v"], st["eta"], st["U"], st["W"]),
                                           (d["v"][..., None], d["eta"][..., None], None, None)]))
        finally:
            ens.close()
    for a, b2 in zip(out[0], out[1]):
        for x, y in zip(a[:2], b2[:2]):
            assert np.array_equal(x, y)
    assert np.array_equal(out[0][0][2], out[1][0][2]) and np.array_equal(out[0][0][3], out[1][0][3])


def _fused_cache(tmp_path):
    """An autotune cache that puts G's member blocks of 4 on the fused stage in
    parity blocks (helm 7) with the y-derivatives in parity blocks tuned (3) and
    the tile shapes fixed, so that every handle below runs the same kernels; its
    whole-step times put the step-by-step stage in parity blocks (helm 8) 1 us
    per step behind, less than the derivatives of a new state cost."""
    p = tmp_path / "tune.txt"
    p.write_text("plane 32 33 32 4 3\nygemm 32 33 32 4 3\n"
                 "helm 32 33 32 4 7   # variant 7 0.2000 ms variant 8 0.2010 ms\nspec_ec 32 33 32 4 4\n"
                 "spec_cta 32 33 32 4 3\nytile 32 33 32 4 16\n")
    return str(p)


@pytest.mark.parametrize("use_graph", [True, False])
def test_short_advance_calls_run_the_step_by_step_stage_of_a_fused_block(tmp_path, use_graph):
    """A block the autotuner put on the fused stage runs, in dns_advance calls of
    one or two steps with page-locked buffers, its step-by-step stage in parity
    blocks (no derivatives of the uploaded state needed): the call equals
    set_state + step + get_state on that stage bit for bit.  The next fused
    step first computes the derivatives of its state (as setting that state
    and stepping does), and a four-step call runs the fused stage."""
    cache = _fused_cache(tmp_path)
    st = _state()
    keys = ("v", "eta", "U", "W")

    def run(nsteps, **kw):
        e = dns.Ensemble([G], precision="mixed", use_graph=use_graph, autotune_cache=cache, **kw)
        try:
            e.set_state(0, *(st[k] for k in keys))
            e.step(nsteps)
            return e.get_state(0)
        finally:
            e.close()

    ens = dns.Ensemble([G], precision="mixed", use_graph=use_graph, autotune_cache=cache)
    try:
        assert dns.dns_kernel_choice(ens.h, 0, "helm") == "fused_eo_ff"
        keep_in = [_pinned(st[k]) for k in keys]
        for nsteps, kw in ((1, dict(helm="simt_eo", ygemm="simt_eo", plane="lines")),
                           (2, dict(helm="simt_eo", ygemm="simt_eo", plane="lines")),
                           (4, {})):
            ref = run(nsteps, **kw)
            keep_out = [_pinned(np.zeros_like(x)) for x in ref]
            dns.dns_advance(ens.h, nsteps, [tuple(_ptr(t) for _, t in keep_in)],
                            [tuple(_ptr(t) for _, t in keep_out)], 0)
            got = [_host(t, x).copy() for (_, t), x in zip(keep_out, ref)]
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), nsteps
        # continue on the fused stage from the state a one-step call left: its
        # derivatives are computed first, as setting that state computes them.  A
        # state read back and set again differs from the device's by the Hermitian
        # projection of the n = 0 column, at FP64 rounding level, which can flip
        # single-precision roundings downstream (measured 7e-9 of the field after
        # two steps); the derivatives of the previous sub-stage's state, which the
        # per-plane arrays held, would be off at O(dt) = 5e-3 of the field.
        dns.dns_advance(ens.h, 1, [tuple(_ptr(t) for _, t in keep_in)], None, 0)
        mid = ens.get_state(0)
        ens.step(2)
        cont = ens.get_state(0)
        e2 = dns.Ensemble([G], precision="mixed", use_graph=use_graph, autotune_cache=cache)
        try:
            e2.set_state(0, *mid)
            e2.step(2)
            want = e2.get_state(0)
        finally:
            e2.close()
        for a, b in zip(cont, want):
            assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
    finally:
        ens.close()
