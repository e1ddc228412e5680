"""Checkpoint files of the binding (host only): save_states / load_states keep
every group description and every state array exactly, None entries included,
and same_groups tells a checkpoint's groups apart from others."""
import numpy as np
import pytest

import dns_synth


@pytest.fixture(scope="module")
def dns():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_12739_gb300 as mod
    return mod


def test_states_round_trip_exactly(dns, tmp_path):
    g1 = dict(flow="poiseuille", mx=16, my=17, mz=16, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=3)
    g2 = dict(flow="couette", mx=0, my=21, mz=16, lx=2 * np.pi, lz=np.pi, re=1000.0, dt=0.02, members=2,
              linear=True, kx_index=1)
    st = dns_synth.make_state(16, 17, 16, g1["lx"], g1["lz"], "poiseuille", 3, 11, 5e-2)
    d = dns_synth.make_disturbances(21, 16, np.pi, 2, 12)
    states = [(st["v"], st["eta"], st["U"], st["W"]), (d["v"][..., None], d["eta"][..., None], None, None)]
    path = str(tmp_path / "ck.npz")
    dns.save_states(path, [g1, g2], states)
    groups, back = dns.load_states(path)
    assert dns.same_groups(groups, [g1, g2])
    for a, b in zip(states, back):
        for x, y in zip(a, b):
            if x is None:
                assert y is None
            else:
                assert x.dtype == y.dtype and np.array_equal(x, y)


def test_same_groups_tells_other_groups_apart(dns):
    g = dict(flow="couette", mx=16, my=17, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=2)
    assert dns.same_groups([g], [dict(g)])
    assert not dns.same_groups([g], [dict(g, members=3)])
    assert not dns.same_groups([g], [dict(g, re=401.0)])
    assert not dns.same_groups([g], [g, g])
