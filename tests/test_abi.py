"""C-ABI library: loads, exports every declared symbol, validates input, and
builds the same operators as the oracle (host only, no GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dns():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_12739_gb300 as mod
    return mod


def _declared():
    txt = open(os.path.join(ROOT, "include", "dns.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dns_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(dns):
    declared = _declared()
    assert len(declared) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", dns.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dns_[a-z_]+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert sorted(dns.EXPORTED) == declared
    for s in declared:
        assert hasattr(dns._lib, s)


def test_build_targets_sm_103a_only(dns):
    from paper_2306_12739_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _g(**kw):
    g = dict(flow="couette", mx=16, my=33, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=1)
    g.update(kw)
    return g


@pytest.mark.parametrize("bad,code", [
    (dict(mx=40), -6), (dict(mz=128), -6), (dict(my=3), -6), (dict(my=200), -6),
    (dict(re=0.0), -1), (dict(dt=-1.0), -1), (dict(members=0), -1), (dict(lx=0.0), -1),
])
def test_invalid_configurations_are_rejected(dns, bad, code):
    with pytest.raises(dns.DnsError) as ei:
        dns.dns_create(dns.make_config([_g(**bad)]), 0)
    assert ei.value.code == code


def test_calls_before_binding_fail_cleanly(dns):
    h = dns.dns_create(dns.make_config([_g()]), 0)
    try:
        with pytest.raises(dns.DnsError) as ei:
            dns.dns_step(h, 1)
        assert ei.value.code == dns.DNS_ERR_INVALID
        assert "not bound" in dns.dns_last_error(h)
        assert dns._lib.dns_bind_workspace(h, ctypes.c_void_p(256), 16) == dns.DNS_ERR_NOMEM
        assert dns._lib.dns_bind_workspace(h, ctypes.c_void_p(3), 1 << 40) == dns.DNS_ERR_INVALID
        assert dns.dns_state_shape(h, 0) == (6, 11, 31, 33)
        with pytest.raises(dns.DnsError):
            dns.dns_state_shape(h, 1)
    finally:
        dns.dns_destroy(h)


@pytest.mark.parametrize("flow,mx,my,mz,lx,lz,re,dt", [
    ("couette", 16, 33, 16, 1.75 * np.pi, 1.2 * np.pi, 400.0, 0.01),
    ("poiseuille", 48, 49, 32, 2 * np.pi, np.pi, 1650.0, 0.005),
])
def test_library_operators_equal_oracle_operators(dns, flow, mx, my, mz, lx, lz, re, dt):
    """The library builds its operators in double-double with LU; the oracle in
    quad with Gauss-Jordan and different derivative formulas.  Rounded to double
    they agree to the last bit."""
    g = _g(flow=flow, mx=mx, my=my, mz=mz, lx=lx, lz=lz, re=re, dt=dt)
    h = dns.dns_create(dns.make_config([g]), 0)
    try:
        ch = oracle.Channel(mx, my, mz, lx, lz, re, dt, flow)
        y, D1, D2, D4, w = dns.dns_export_grid(h, 0, my)
        assert np.array_equal(y, ch.y) and np.array_equal(D2, ch.D2) and np.array_equal(D4, ch.D4c)
        assert np.abs(D1 - ch.D1).max() < 1e-30 + 1e-16 * np.abs(ch.D1).max()
        assert np.array_equal(w, ch.w)
        for hi, hv in enumerate((0.5, 1.0)):
            for am in range(ch.Kz + 1):
                for n in range(ch.Kx + 1):
                    got = dns.dns_export_operators(h, 0, hi, am * (ch.Kx + 1) + n, my - 2)
                    for a, b in zip(got, ch.ops[hv]):
                        assert np.array_equal(a, b[ch.Kz + am, n])
    finally:
        dns.dns_destroy(h)
