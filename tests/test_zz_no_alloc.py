"""dns_stats_noalloc, the statistics entry point for callers that cannot
allocate device memory (e.g. inside an embedding runtime's step callback),
against dns_stats through the C ABI.  Collected last on purpose."""
import numpy as np
import pytest

import dns_synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_12739_gb300 as dns  # noqa: E402

KEYS = ("e_total", "e_pert", "tau_bottom", "tau_top", "bulk_flux", "gamma", "max_div", "nonfinite")


def _compare_two_calls_in_a_row(ens, members, group=0):
    out = torch.empty((members, 8), dtype=torch.float64, device="cuda")
    for _ in range(2):
        ens.step(2)
        ref = ens.stats(group)                  # existing entry point (synchronises)
        with torch.cuda.stream(ens.stream):
            out.fill_(float("nan"))             # every value must be written by the call
        dns.dns_stats_noalloc(ens.h, group, out.data_ptr())
        ens.stream.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        for i, k in enumerate(KEYS):
            want = np.asarray(ref[k], dtype=np.float64)
            if k == "max_div":
                assert np.all(np.abs(got[:, i] - want) <= 1e-13), k
            else:
                assert np.all(np.abs(got[:, i] - want) <= 1e-12 * max(1.0, np.abs(want).max())), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stats_noalloc_matches_dns_stats_on_two_calls_in_a_row(precision):
    g = dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=3)
    st = dns_synth.make_state(32, 33, 32, g["lx"], g["lz"], "poiseuille", 3, 61, 5e-2)
    ens = dns.Ensemble([g], precision=precision)
    try:
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        _compare_two_calls_in_a_row(ens, 3)
    finally:
        ens.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stats_noalloc_over_several_member_blocks(precision):
    # 40 independent members run as four blocks of 10: each block writes its
    # rows at its own offset of the output and reuses the one array after the
    # block before it on the stream
    E = 40
    g = dict(flow="couette", mx=16, my=25, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=E,
             member_block=10)
    st = dns_synth.make_state(16, 25, 16, g["lx"], g["lz"], "couette", E, 71, np.linspace(1e-2, 5e-2, E))
    ens = dns.Ensemble([g], precision=precision)
    try:
        ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
        _compare_two_calls_in_a_row(ens, E)
    finally:
        ens.close()


def test_stats_noalloc_of_a_linear_group():
    my, mz, lz, E = 33, 32, np.pi, 3
    g = dict(flow="couette", mx=0, my=my, mz=mz, lx=2 * np.pi, lz=lz, re=1000.0, dt=0.02, members=E,
             linear=True, kx_index=1)
    b = dns_synth.make_base_flow(my, mz, lz, "couette", 5, streak=0.3, roll=0.03)
    d = dns_synth.make_disturbances(my, mz, lz, E, 105)
    ens = dns.Ensemble([g], precision="fp64")
    try:
        ens.set_base_flow(0, b["U"], b["V"], b["W"])
        ens.set_state(0, d["v"][..., None], d["eta"][..., None])
        _compare_two_calls_in_a_row(ens, E)
    finally:
        ens.close()


def test_stats_noalloc_rejects_a_group_larger_than_its_array():
    # 127 interior planes; 1400 members need 1066800 > 2^20 partials.  A shared-mean
    # group is one block (independent members would run in blocks of about 16)
    g = dict(flow="couette", mx=16, my=129, mz=16, lx=2 * np.pi, lz=np.pi, re=400.0, dt=0.01, members=1400,
             shared_mean=True)
    cfg = dns.make_config([g])
    h = dns.dns_create(cfg, 0)
    try:
        n = dns.dns_workspace_size(h)
        ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        dns.dns_bind_workspace(h, (ws.data_ptr() + 255) & ~255, n)
        out = torch.empty((1400, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(dns.DnsError) as ei:
            dns.dns_stats_noalloc(h, 0, out.data_ptr())
        assert ei.value.code == dns.DNS_ERR_INVALID
        assert "fixed array" in str(ei.value)
    finally:
        dns.dns_destroy(h)
