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
    (dict(member_block=-1), -1),
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


def test_integer_pipe_conversions_round_like_ieee(dns):
    """The mixed-precision kernels convert their FP64 state with integer
    operations (binary64 -> binary32 round to nearest even; binary32 ->
    binary64 exact); the host run of the same code must agree with IEEE
    conversions on random values over the whole normal range, on exact ties in
    both directions, and on signed zeros, infinities and NaN; magnitudes below
    2^-126 flush to signed zero."""
    import numpy as np
    rng = np.random.default_rng(7)
    n = 200000
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-125, 127, n)
    d = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)
    # exact ties: a binary32 value plus half an ulp, with even and odd last bits
    base = np.float32(rng.uniform(1.0, 2.0, 5000)).astype(np.float64)
    ulp = np.spacing(np.float32(base)).astype(np.float64)
    ties = np.concatenate([base + 0.5 * ulp, -(base + 0.5 * ulp), base + 0.5 * ulp * (1 + 2 ** -20)])
    special = np.array([0.0, -0.0, np.inf, -np.inf, 3.4e38, -3.4e38, 1.1754943508222875e-38,
                        np.finfo(np.float32).max.astype(np.float64), 1e-300, -1e-300, 2.0 ** -127])
    d = np.concatenate([d, ties, special])
    f = np.float32(rng.standard_normal(d.size)) * np.float32(10.0) ** rng.integers(-30, 30, d.size).astype(np.float32)
    f[:4] = [0.0, -0.0, np.inf, -np.inf]
    f_out, d_out = dns.convert_selftest(d, f)
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)
    tiny = np.abs(d) < 2.0 ** -126
    ref[tiny] = np.copysign(np.float32(0.0), d[tiny]).astype(np.float32)
    assert np.array_equal(f_out.view(np.uint32), ref.view(np.uint32))
    ref_d = f.astype(np.float64)
    sub = (np.abs(f) < np.finfo(np.float32).tiny) & (f != 0)
    ref_d[sub] = np.copysign(0.0, f[sub])
    assert np.array_equal(d_out.view(np.uint64), ref_d.view(np.uint64))
    fn, _ = dns.convert_selftest(np.array([np.nan]), np.array([np.nan], dtype=np.float32))
    assert np.isnan(fn[0])


def test_rotational_form_is_refused_where_no_kernel_has_it(dns):
    g = dict(flow="couette", mx=128, my=33, mz=128, lx=2 * np.pi, lz=np.pi, re=400.0, dt=0.01, members=1,
             form="rotational")
    for prec in ("fp64", "mixed"):
        with pytest.raises(dns.DnsError) as ei:
            dns.dns_create(dns.make_config([g], precision=prec), 0)
        assert ei.value.code == dns.DNS_ERR_UNSUPPORTED
    bad = dict(g, mx=32, mz=32)
    cfg = dns.make_config([bad])
    cfg.groups[0].nonlinear_form = 5
    with pytest.raises(dns.DnsError) as ei:
        dns.dns_create(cfg, 0)
    assert ei.value.code == dns.DNS_ERR_INVALID


def _lin_group(**kw):
    g = dict(flow="couette", mx=0, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1000.0, dt=0.04, members=3,
             linear=True, kx_index=2)
    g.update(kw)
    return g


def test_linear_groups_validate_and_build_the_single_kx_operators(dns):
    for bad in (dict(kx_index=0), dict(shared_mean=True), dict(form="rotational")):
        with pytest.raises(dns.DnsError) as ei:
            dns.dns_create(dns.make_config([_lin_group(**bad)]), 0)
        assert ei.value.code == dns.DNS_ERR_INVALID
    with pytest.raises(dns.DnsError) as ei:
        dns.dns_create(dns.make_config([_lin_group(mz=40)]), 0)
    assert ei.value.code == dns.DNS_ERR_UNSUPPORTED
    g = _lin_group(members=40)                     # one block whatever the size
    h = dns.dns_create(dns.make_config([g]), 0)
    try:
        assert dns.dns_state_shape(h, 0) == (1, 21, 31, 33)
        from oracle.linear import Linear
        z = np.zeros((33, 32))
        lin = Linear(33, 32, g["lx"], g["lz"], g["re"], g["dt"], 2, z, z, z)
        for hi, hv in enumerate((0.5, 1.0)):
            for am in range(lin.Kz + 1):
                got = dns.dns_export_operators(h, 0, hi, am, 31)
                for a, b in zip(got, lin.ops[hv]):
                    assert np.array_equal(a, b[lin.Kz + am])
        for fn in (lambda: dns.dns_set_direction(h, 0, 1), lambda: dns.dns_orthonormalize(h, 0)):
            with pytest.raises(dns.DnsError) as ei:
                fn()
            assert "not bound" in str(ei.value)
    finally:
        dns.dns_destroy(h)


def test_forcing_calls_before_binding_fail_cleanly(dns):
    """Calls before binding fail cleanly; the structures themselves are
    compared with the oracle's in the GPU tests (the call needs a bound
    workspace, which needs device memory)."""
    g = _g(my=33)
    h = dns.dns_create(dns.make_config([g]), 0)
    try:
        with pytest.raises(dns.DnsError) as ei:
            dns.dns_set_stochastic_forcing(h, 0, 1, 4, 1e-3, 7)
        assert "not bound" in str(ei.value)
        with pytest.raises(dns.DnsError):
            dns.dns_export_forcing(h, 0, 0, 4, 31)
    finally:
        dns.dns_destroy(h)


def test_state_transfer_and_advance_calls_before_binding_fail_cleanly(dns):
    h = dns.dns_create(dns.make_config([_g(members=2)]), 0)
    try:
        for call in (lambda: dns.dns_advance(h, 1, None, None, 0),
                     lambda: dns.dns_set_state(h, 0, 0, 1, 8, 8, 8, 8, 0),
                     lambda: dns.dns_get_state(h, 0, 0, 1, 8, 8, 8, 8, 0)):
            with pytest.raises(dns.DnsError) as ei:
                call()
            assert ei.value.code == dns.DNS_ERR_INVALID
            assert "not bound" in dns.dns_last_error(h)
    finally:
        dns.dns_destroy(h)


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "dns.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
int main(void) {
    printf("dns_stats_t size %zu\n", sizeof(dns_stats_t));
    F(dns_stats_t, e_total) F(dns_stats_t, e_pert) F(dns_stats_t, tau_bottom) F(dns_stats_t, tau_top)
    F(dns_stats_t, bulk_flux) F(dns_stats_t, gamma) F(dns_stats_t, max_div) F(dns_stats_t, nonfinite)
    F(dns_stats_t, reserved) F(dns_stats_t, cfl)
    printf("dns_state_in size %zu\n", sizeof(dns_state_in));
    F(dns_state_in, v_hat) F(dns_state_in, eta_hat) F(dns_state_in, U00) F(dns_state_in, W00)
    printf("dns_state_out size %zu\n", sizeof(dns_state_out));
    F(dns_state_out, v_hat) F(dns_state_out, eta_hat) F(dns_state_out, U00) F(dns_state_out, W00)
    printf("dns_group_desc size %zu\n", sizeof(dns_group_desc));
    F(dns_group_desc, flow) F(dns_group_desc, mx) F(dns_group_desc, my) F(dns_group_desc, mz)
    F(dns_group_desc, lx) F(dns_group_desc, lz) F(dns_group_desc, re) F(dns_group_desc, dt)
    F(dns_group_desc, u_wall) F(dns_group_desc, bulk_flux) F(dns_group_desc, members)
    F(dns_group_desc, shared_mean) F(dns_group_desc, nonlinear_form) F(dns_group_desc, member_block)
    F(dns_group_desc, linear) F(dns_group_desc, kx_index)
    printf("dns_config size %zu\n", sizeof(dns_config));
    F(dns_config, n_groups) F(dns_config, groups) F(dns_config, precision) F(dns_config, use_graph)
    F(dns_config, persistent) F(dns_config, barrier_timeout_ns) F(dns_config, autotune_cache)
    F(dns_config, ygemm) F(dns_config, plane) F(dns_config, helm)
    return 0;
}
"""


def test_python_struct_mirrors_match_the_c_header(dns, tmp_path):
    """Every struct the binding passes across the ABI has the header's size and
    field offsets (compiled with the host C compiler against include/dns.h)."""
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        t, f, v = line.split()
        c[(t, f)] = int(v)
    for name in ("dns_stats_t", "dns_state_in", "dns_state_out", "dns_group_desc", "dns_config"):
        cls = getattr(dns, name)
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(name, field)], (name, field)


@pytest.mark.parametrize("kw,word", [(dict(ygemm="bogus"), "ygemm"), (dict(plane="fast"), "plane"),
                                     (dict(helm="x"), "helm"), (dict(precision="fp16"), "precision")])
def test_unknown_names_are_rejected_with_the_choices(dns, kw, word):
    with pytest.raises(ValueError) as ei:
        dns.make_config([_g()], **kw)
    assert word in str(ei.value) and "choices" in str(ei.value)
    with pytest.raises(ValueError):
        dns.make_config([_g(flow="channel")])


def test_autotune_cache_path_may_come_from_the_environment(dns, monkeypatch, tmp_path):
    path = str(tmp_path / "tune.txt")
    monkeypatch.setenv("DNS_AUTOTUNE_CACHE", path)
    assert dns.make_config([_g()]).autotune_cache == path.encode()
    assert dns.make_config([_g()], autotune_cache="other").autotune_cache == b"other"
    monkeypatch.delenv("DNS_AUTOTUNE_CACHE")
    assert dns.make_config([_g()]).autotune_cache is None


def test_kernel_choice_names_are_the_request_names(dns, monkeypatch):
    """Every kernel variant a caller can request reads back under the same name
    (the C call faked: it reports the requested numbers)."""
    import ctypes

    class Fake:
        value = (0, 0, 0)

        def dns_kernel_choice(self, h, group, c, p, m):
            for ref, v in zip((c, p, m), self.value):
                ctypes.cast(ref, ctypes.POINTER(ctypes.c_int))[0] = v
            return 0

    fake = Fake()
    monkeypatch.setattr(dns, "_lib", fake)
    for which, table in (("ygemm", dns._YGEMM), ("plane", dns._PLANE), ("helm", dns._HELM)):
        for name, num in table.items():
            if num == 0:
                continue
            fake.value = tuple(num if w == which else 1 for w in ("ygemm", "plane", "helm"))
            assert dns.dns_kernel_choice(None, 0, which) == name, (which, name)
    fake.value = (1, 4, 1)
    assert dns.dns_kernel_choice(None, 0, "plane") == "linear"

