"""The bounds-checked debug build (libdns_check.so, compiled with -DDNS_CHECK):
every index of the hot-path kernels' global accesses (and of the fused stage's
shared-memory vectors) is checked; a failure records the kernel and the index
in the device status word, skips the access and is reported by the next
synchronising call.  A small-grid parity subset runs under it in a child
process (the library is chosen when the package is imported) and must finish
without a report and with the results of the normal build."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, groups, precision, pins, steps, forcing)
CASES = [
    ("fused_d2tc", [dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                         members=3)], "mixed", dict(helm="fused"), 3, None),
    ("fused_chunks", [dict(flow="couette", mx=16, my=21, mz=48, lx=2 * np.pi, lz=np.pi, re=400.0, dt=0.005,
                           members=20, member_block=20)], "mixed", dict(helm="fused"), 3, None),
    ("fused_d2v_inside", [dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                               members=6, member_block=6)], "mixed", dict(helm="fused_d2v"), 3, None),
    ("fused_parity_ff", [dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                              members=6, member_block=6)], "mixed", dict(helm="fused_eo_ff"), 3, None),
    ("fused_parity", [dict(flow="couette", mx=16, my=21, mz=16, lx=2 * np.pi, lz=np.pi, re=400.0, dt=0.005,
                           members=3)], "mixed", dict(helm="fused_eo"), 3, None),
    ("fused_floatfloat", [dict(flow="poiseuille", mx=32, my=97, mz=16, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                               members=2)], "mixed", dict(helm="fused"), 3, None),
    ("yderiv_parity", [dict(flow="poiseuille", mx=32, my=34, mz=16, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                            members=5)], "mixed", dict(helm="simt", ygemm="simt_eo"), 3, None),
    ("step_parity", [dict(flow="couette", mx=16, my=21, mz=16, lx=2 * np.pi, lz=np.pi, re=400.0, dt=0.005,
                          members=3)], "mixed", dict(helm="simt_eo"), 3, (1, 2, 1e-3, 5)),
    ("chain_tc", [dict(flow="couette", mx=32, my=49, mz=32, lx=1.75 * np.pi, lz=1.2 * np.pi, re=500.0, dt=0.01,
                       members=8)], "mixed", dict(helm="simt", ygemm="tc"), 3, None),
    ("fp64", [dict(flow="couette", mx=16, my=33, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01,
                   members=2)], "fp64", {}, 3, None),
    ("forced", [dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005,
                     members=4)], "mixed", dict(helm="fused"), 3, (1, 4, 1e-3, 7)),
]

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import dns_synth
import paper_2306_12739_gb300 as dns
assert dns.dns_checked_build() == 1, "the child did not load the checked build"
cases = json.loads({cases!r})
out = {{}}
for name, groups, prec, pins, steps, forcing in cases:
    g = groups[0]
    st = dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"], 11, 5e-2)
    ens = dns.Ensemble(groups, precision=prec, **pins)
    try:
        if name == "fused_d2tc":
            rc = dns.dns_selftest_bounds(ens.h)
            out["selftest_rc"] = rc
            out["selftest_msg"] = dns.dns_last_error(ens.h)
        if forcing is not None:
            ens.set_stochastic_forcing(0, *forcing)
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        ens.step(steps)
        res = ens.get_state(0)            # synchronises: a bounds report raises here
        # the transfer kernels (pack, unpack) through dns_advance
        res2 = ens.advance(1, [res])[0]
        np.savez({tmp!r} + "/" + name + ".npz", *res, *res2)
    finally:
        ens.close()
print(json.dumps(out))
"""


def _build_checked():
    spec = importlib.util.spec_from_file_location("_dns_build_checked", os.path.join(ROOT, "paper_2306_12739_gb300",
                                                                                    "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build(checked=True)


def test_checked_build_runs_the_parity_subset_without_a_report_and_matches_the_normal_build(tmp_path):
    import dns_synth
    _build_checked()
    code = CHILD.format(root=ROOT, cases=json.dumps(CASES), tmp=str(tmp_path))
    env = dict(os.environ, DNS_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    # the self-test's failing check (kernel 1, index 12345) is reported, and the
    # handle kept working afterwards (the parity runs above used it)
    assert info["selftest_rc"] == dns.DNS_ERR_CUDA
    assert "bounds check failed: kernel 1, index 12345" in info["selftest_msg"]
    for name, groups, prec, pins, steps, forcing in CASES:
        g = groups[0]
        st = dns_synth.make_state(g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["flow"], g["members"], 11, 5e-2)
        ens = dns.Ensemble(groups, precision=prec, **pins)
        try:
            if forcing is not None:
                ens.set_stochastic_forcing(0, *forcing)
            ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
            ens.step(steps)
            ref = ens.get_state(0)
            ref2 = ens.advance(1, [ref])[0]
        finally:
            ens.close()
        got = np.load(str(tmp_path / (name + ".npz")))
        arrays = [got["arr_%d" % i] for i in range(8)]
        tol = 1e-12 if prec == "fp64" else 1e-6
        for a, b in zip(arrays, list(ref) + list(ref2)):
            assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300), name


def test_normal_build_has_no_checks():
    assert dns.dns_checked_build() == 0
    g = dict(flow="couette", mx=16, my=33, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=1)
    ens = dns.Ensemble([g], precision="fp64")
    try:
        assert dns.dns_selftest_bounds(ens.h) == dns.DNS_OK
    finally:
        ens.close()
