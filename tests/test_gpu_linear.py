"""Linearised disturbance groups on the GPU (through the C ABI) against the
oracle (oracle.linear): forward and adjoint steps, the energy statistics,
energy-norm Gram-Schmidt and whole forward-adjoint optimal-growth sweeps, in
FP64; the mixed path against FP64; member independence."""
import numpy as np
import pytest

import dns_synth
from oracle.linear import Linear

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

PINS = (dict(ygemm="simt", helm="simt"), dict(ygemm="tc", helm="simt"), dict(ygemm="simt", helm="tc"),
        dict(ygemm="tc", helm="tc"), dict(ygemm="tc", helm="persist"), dict(ygemm="simt_eo", helm="simt"))


def lgroup(my, mz, lz, re, dt, n, E):
    return dict(flow="couette", mx=0, my=my, mz=mz, lx=2 * np.pi, lz=lz, re=re, dt=dt, members=E,
                linear=True, kx_index=n)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _ens(groups, bases, prec="fp64", **kw):
    ens = dns.Ensemble(groups, precision=prec, **kw)
    for gi, b in enumerate(bases):
        ens.set_base_flow(gi, b["U"], b["V"], b["W"])
    return ens


def _get(ens, gi):
    v, e, _, _ = ens.get_state(gi)
    return v[..., 0], e[..., 0]


def _case(my, mz, lz, n, E, seed, flow="couette"):
    b = dns_synth.make_base_flow(my, mz, lz, flow, seed, streak=0.3, roll=0.03)
    d = dns_synth.make_disturbances(my, mz, lz, E, 100 + seed)
    return b, d


@pytest.mark.parametrize("my,mz,n,E,flow", [(33, 32, 1, 3, "couette"), (25, 16, 2, 2, "poiseuille"),
                                            (49, 48, 3, 4, "couette"), (65, 64, 1, 3, "poiseuille"),
                                            (21, 128, 2, 2, "couette"), (129, 16, 1, 2, "couette")])
def test_linear_fp64_forward_and_adjoint_steps_match_the_oracle(my, mz, n, E, flow):
    lz, re, dt = np.pi, 1000.0, 0.02
    b, d = _case(my, mz, lz, n, E, 7, flow)
    lin = Linear(my, mz, 2 * np.pi, lz, re, dt, n, b["U"], b["V"], b["W"])
    ens = _ens([lgroup(my, mz, lz, re, dt, n, E)], [b])
    try:
        ens.set_state(0, d["v"][..., None], d["eta"][..., None])
        ens.step(4)
        ref = lin.step((d["v"], d["eta"]), 4)
        for a, r in zip(_get(ens, 0), ref):
            assert rel(a, r) < 1e-11
        ens.set_direction(True)
        ens.step(4)
        ref2 = lin.step(ref, 4, adjoint=True)
        got2 = _get(ens, 0)
        for a, r in zip(got2, ref2):
            assert rel(a, r) < 1e-11
        assert rel(got2[0], lin.step(ref, 4)[0]) > 1e-6    # the adjoint is a different map
        st = ens.stats(0)
        assert np.allclose(st["e_pert"], lin.energy(ref2), rtol=1e-11, atol=0)
        assert np.all(st["e_total"] == st["e_pert"]) and np.all(st["bulk_flux"] == 0.0)
    finally:
        ens.close()


def test_linear_base_flow_matters_and_zero_base_flow_is_pure_viscous_decay():
    my, mz, lz, re, dt, n, E = 33, 32, np.pi, 1000.0, 0.02, 1, 2
    b, d = _case(my, mz, lz, n, E, 3)
    z = {k: np.zeros_like(a) for k, a in b.items()}
    lin0 = Linear(my, mz, 2 * np.pi, lz, re, dt, n, z["U"], z["V"], z["W"])
    ens = dns.Ensemble([lgroup(my, mz, lz, re, dt, n, E)], precision="fp64")   # base flow never set
    try:
        ens.set_state(0, d["v"][..., None], d["eta"][..., None])
        ens.step(3)
        ref = lin0.step((d["v"], d["eta"]), 3)
        for a, r in zip(_get(ens, 0), ref):
            assert rel(a, r) < 1e-11
        e0 = lin0.energy((d["v"], d["eta"]))
        assert np.all(ens.stats(0)["e_pert"] < e0)
        ens.set_base_flow(0, b["U"], b["V"], b["W"])
        ens.set_state(0, d["v"][..., None], d["eta"][..., None])
        ens.step(3)
        assert rel(_get(ens, 0)[0], ref[0]) > 1e-3
    finally:
        ens.close()


def test_linear_gram_schmidt_matches_the_oracle():
    my, mz, lz, E = 33, 32, np.pi, 6
    b, d = _case(my, mz, lz, 1, E, 11)
    d["v"][4] = d["v"][0] - 0.5j * d["v"][2] + 1e-3 * d["v"][4]
    d["eta"][4] = d["eta"][0] - 0.5j * d["eta"][2] + 1e-3 * d["eta"][4]
    lin = Linear(my, mz, 2 * np.pi, lz, 1000.0, 0.02, 1, b["U"], b["V"], b["W"])
    ens = _ens([lgroup(my, mz, lz, 1000.0, 0.02, 1, E)], [b])
    try:
        ens.set_state(0, d["v"][..., None], d["eta"][..., None])
        r = ens.orthonormalize(0)
        got = _get(ens, 0)
        Q, rr = lin.orthonormalize((d["v"], d["eta"]))
        assert np.all(np.abs(r - rr) < 1e-12 * np.sqrt(lin.energy((d["v"], d["eta"]))))
        # vector 4 lost three digits to cancellation in both; compare at that level
        for a, q in zip(got, Q):
            assert rel(a, q) < 1e-9
            assert rel(np.delete(a, 4, 0), np.delete(q, 4, 0)) < 1e-12
        assert np.max(np.abs(lin.inner(got, got) - np.eye(E))) < 1e-12
        assert np.allclose(ens.stats(0)["e_pert"], 1.0, rtol=1e-12, atol=0)
    finally:
        ens.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_optimal_sweeps_of_two_wavenumbers_match_the_oracle(use_graph):
    """Two linear groups (kx index 1 and 2, different sizes) in one handle: whole
    forward-adjoint-Gram-Schmidt iterations, states and gains."""
    my, mz, lz, re, dt, nsteps = 33, 32, np.pi, 1000.0, 0.04, 10
    cases = [(1, 3, 21), (2, 2, 22)]
    groups, bases, lins, X = [], [], [], []
    for n, E, seed in cases:
        b, d = _case(my, mz, lz, n, E, seed)
        groups.append(lgroup(my, mz, lz, re, dt, n, E))
        bases.append(b)
        lins.append(Linear(my, mz, 2 * np.pi, lz, re, dt, n, b["U"], b["V"], b["W"]))
        X.append((d["v"], d["eta"]))
    ens = _ens(groups, bases, use_graph=use_graph)
    try:
        for gi, x in enumerate(X):
            ens.set_state(gi, x[0][..., None], x[1][..., None])
        for it in range(2):
            gains = ens.optimal_sweep(nsteps)
            for gi, lin in enumerate(lins):
                X[gi], r = lin.sweep(X[gi], nsteps)
                assert np.allclose(gains[gi], r, rtol=1e-11, atol=0), (it, gi)
                for a, q in zip(_get(ens, gi), X[gi]):
                    assert rel(a, q) < 1e-10
        assert ens.launches() > 0
    finally:
        ens.close()


@pytest.mark.parametrize("pin", PINS, ids=["simt", "tc_ygemm", "tc_helm", "tc_both", "persist_helm", "eo_ygemm"])
def test_linear_mixed_matches_fp64_over_50_steps(pin):
    my, mz, lz, re, dt, n, E = 65, 64, np.pi, 3000.0, 0.04, 1, 6
    b, d = _case(my, mz, lz, n, E, 5)
    g = lgroup(my, mz, lz, re, dt, n, E)
    out = {}
    for prec in ("fp64", "mixed"):
        ens = _ens([g], [b], prec=prec, **(pin if prec == "mixed" else {}))
        try:
            ens.set_state(0, d["v"][..., None], d["eta"][..., None])
            ens.step(50)
            fwd = _get(ens, 0)
            ens.set_direction(True)
            ens.step(50)
            out[prec] = fwd + _get(ens, 0)
            if prec == "mixed":
                assert dns.dns_kernel_choice(ens.h, 0, "ygemm") == pin["ygemm"]
                assert dns.dns_kernel_choice(ens.h, 0, "helm") == pin["helm"]
                assert dns.dns_kernel_choice(ens.h, 0, "plane") == "linear"
        finally:
            ens.close()
    for a, r in zip(out["mixed"], out["fp64"]):
        assert rel(a, r) < 1e-5, rel(a, r)


@pytest.mark.parametrize("prec,pin", [("fp64", {}), ("mixed", dict(ygemm="tc", helm="tc")),
                                      ("mixed", dict(ygemm="simt", helm="simt"))])
def test_a_disturbance_evolves_bitwise_alone_as_in_its_ensemble(prec, pin):
    my, mz, lz, re, dt, n, E = 33, 32, np.pi, 1000.0, 0.04, 2, 5
    b, d = _case(my, mz, lz, n, E, 9)
    res = []
    for sel in (slice(0, E), slice(3, 4)):
        ens = _ens([lgroup(my, mz, lz, re, dt, n, sel.stop - sel.start)], [b], prec=prec, use_graph=True, **pin)
        try:
            ens.set_state(0, d["v"][sel][..., None], d["eta"][..., None][sel])
            ens.step(3)
            ens.set_direction(True)
            ens.step(2)
            res.append(_get(ens, 0))
        finally:
            ens.close()
    for a, b_ in zip(res[0], res[1]):
        assert np.array_equal(a[3:4], b_)


def test_parity_block_request_runs_the_natural_order_apply_in_a_linear_group():
    """The operators of a linearised group include the base flow, which need
    not be symmetric in y: a request for the parity-block step-by-step stage
    runs the natural-order one there, bit for bit the same as asking for it."""
    my, mz, lz, re, dt, n, E = 33, 32, np.pi, 1000.0, 0.04, 1, 3
    b, d = _case(my, mz, lz, n, E, 13)
    out = []
    for helm in ("simt_eo", "simt"):
        ens = _ens([lgroup(my, mz, lz, re, dt, n, E)], [b], prec="mixed", ygemm="simt", helm=helm)
        try:
            assert dns.dns_kernel_choice(ens.h, 0, "helm") == "simt"
            ens.set_state(0, d["v"][..., None], d["eta"][..., None])
            ens.step(3)
            out.append(_get(ens, 0))
        finally:
            ens.close()
    for a, c in zip(out[0], out[1]):
        assert np.array_equal(a, c)
