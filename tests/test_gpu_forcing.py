"""Stochastic forcing on the GPU (through the C ABI) against the oracle
(oracle.forcing): structures, forced FP64 steps (independent and shared-mean
ensembles), graph replay and member blocks bitwise, mixed vs FP64, switching
off and restarting the noise."""
import numpy as np
import pytest

import dns_synth
import oracle
from oracle.forcing import StochasticForcing

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

FIELDS = ("v", "eta", "U", "W")


def group(flow, mx, my, mz, re, dt, E, **kw):
    g = dict(flow=flow, mx=mx, my=my, mz=mz, lx=2 * np.pi, lz=np.pi, re=re, dt=dt, members=E)
    g.update(kw)
    return g


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _state(g, seed, amp=2e-2):
    st = dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"], seed, amp,
                              n_max=3, m_max=3)
    if g.get("shared_mean"):
        for k in ("v", "eta"):
            st[k][:, :, :, 0] = st[k][:, :, :, 0].mean(axis=0)[None]
    return st


def _run(g, st, nsteps, forcing, precision="fp64", **kw):
    ens = dns.Ensemble([g], precision=precision, **kw)
    try:
        ens.set_state(0, *(st[k] for k in FIELDS))
        if forcing is not None:
            ens.set_stochastic_forcing(0, *forcing)
        ens.step(nsteps)
        return ens.get_state(0)
    finally:
        ens.close()


def test_forcing_structures_equal_the_oracle():
    g = group("couette", 32, 33, 32, 1000.0, 0.01, 2)
    ch = oracle.Channel(32, 33, 32, g["lx"], g["lz"], g["re"], g["dt"], "couette")
    sf = StochasticForcing(ch, 2, 6, 1e-3, 3)
    ens = dns.Ensemble([g], precision="fp64")
    try:
        ens.set_stochastic_forcing(0, 2, 6, 1e-3, 3)
        for mi in range(2 * ch.Kz + 1):
            f, lam = dns.dns_export_forcing(ens.h, 0, mi, 6, ch.nyi)
            assert rel(f, sf.f[mi]) < 1e-12 and rel(lam, sf.lam[mi]) < 1e-14
        with pytest.raises(dns.DnsError):
            ens.set_stochastic_forcing(0, 11, 4, 1e-3, 3)          # Kx = 10
        with pytest.raises(dns.DnsError):
            ens.set_stochastic_forcing(0, 1, 17, 1e-3, 3)          # at most 16 structures
    finally:
        ens.close()


@pytest.mark.parametrize("flow,mx,my,mz,E,n,neig", [("couette", 16, 33, 16, 3, 1, 4),
                                                   ("poiseuille", 32, 25, 48, 2, 3, 5),
                                                   ("couette", 32, 33, 32, 5, 1, 4)])
def test_fp64_forced_steps_match_the_oracle(flow, mx, my, mz, E, n, neig):
    g = group(flow, mx, my, mz, 1000.0, 0.01, E)
    st = _state(g, 40)
    ch = oracle.Channel(mx, my, mz, g["lx"], g["lz"], g["re"], g["dt"], flow)
    ch.stochastic = StochasticForcing(ch, n, neig, 1e-3, 99)
    ref = ch.step(tuple(st[k] for k in FIELDS), 4)
    got = _run(g, st, 4, (n, neig, 1e-3, 99))
    for a, b, k in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-11, k
    plain = _run(g, st, 4, None)
    assert rel(got[0][:, :, :, n], plain[0][:, :, :, n]) > 1e-3          # the forcing acts


def test_fp64_forced_shared_mean_ensemble_matches_the_oracle():
    """The paper's S3T configuration: members share the kx = 0 flow and are
    forced stochastically at kx / a = 1."""
    g = group("couette", 32, 33, 32, 1000.0, 0.01, 4, shared_mean=True)
    st = _state(g, 50)
    ch = oracle.Channel(32, 33, 32, g["lx"], g["lz"], g["re"], g["dt"], "couette", shared_mean=True)
    ch.stochastic = StochasticForcing(ch, 1, 4, 2e-3, 5)
    ref = ch.step(tuple(st[k] for k in FIELDS), 3)
    got = _run(g, st, 3, (1, 4, 2e-3, 5))
    for a, b, k in zip(got, ref, FIELDS):
        assert rel(a, b) < 1e-11, k
    assert np.array_equal(got[2][0], got[2][3])                           # the mean stays shared


@pytest.mark.parametrize("precision,pin", [("fp64", {}), ("mixed", dict(ygemm="tc", plane="lines", helm="simt")),
                                           ("mixed", dict(plane="lines", helm="fused")),
                                           ("mixed", dict(ygemm="tc", plane="lines", helm="simt_eo"))])
def test_forced_graph_replay_and_member_blocks_are_bitwise_invisible(precision, pin):
    g = group("couette", 16, 33, 16, 400.0, 0.01, 40)
    st = _state(g, 60)
    forcing = (2, 3, 5e-3, 11)
    eager_one = _run(dict(g, member_block=40), st, 3, forcing, precision, **pin)
    graph_blocks = _run(dict(g, member_block=8), st, 3, forcing, precision, use_graph=True, **pin)
    for a, b in zip(eager_one, graph_blocks):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("pin", [dict(ygemm="tc", plane="lines", helm="simt"), dict(helm="fused"),
                                 dict(ygemm="tc", plane="lines", helm="simt_eo")])
def test_mixed_forced_run_matches_fp64_over_50_steps(pin):
    """Every step draws new noise (the step counter advances once per step in
    the step-by-step and in the fused stage alike)."""
    g = group("poiseuille", 32, 33, 32, 1650.0, 0.005, 6)
    st = _state(g, 70, amp=5e-2)
    forcing = (1, 4, 1e-3, 123)
    a = _run(g, st, 50, forcing, "fp64")
    b = _run(g, st, 50, forcing, "mixed", **pin)
    scale = max(np.abs(a[2]).max(), np.abs(a[3]).max())
    for x, y, k in zip(b, a, FIELDS):
        err = np.max(np.abs(x - y)) / (scale if k in ("U", "W") else np.max(np.abs(y)))
        assert err < 1e-6, (k, err)


def test_zero_rate_is_unforced_and_setting_the_forcing_restarts_the_noise():
    g = group("couette", 16, 33, 16, 400.0, 0.01, 3)
    st = _state(g, 80)
    off = _run(g, st, 3, (1, 4, 0.0, 1))
    plain = _run(g, st, 3, None)
    for a, b in zip(off, plain):
        assert np.array_equal(a, b)
    ens = dns.Ensemble([g], precision="fp64", use_graph=True)
    try:
        outs = []
        for _ in range(2):
            ens.set_state(0, *(st[k] for k in FIELDS))
            ens.set_stochastic_forcing(0, 1, 4, 1e-3, 21)
            ens.step(3)
            outs.append(ens.get_state(0))
        for a, b in zip(*outs):
            assert np.array_equal(a, b)
        ens.step(1)                                   # a fourth step draws new noise
        assert not np.array_equal(ens.get_state(0)[0], outs[1][0])
    finally:
        ens.close()
