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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stats_noalloc_matches_dns_stats_on_two_calls_in_a_row(precision):
    g = dict(flow="poiseuille", mx=32, my=33, mz=32, lx=2 * np.pi, lz=np.pi, re=1650.0, dt=0.005, members=3)
    st = dns_synth.make_state(32, 33, 32, g["lx"], g["lz"], "poiseuille", 3, 61, 5e-2)
    ens = dns.Ensemble([g], precision=precision)
    ens.set_state(0, st["v"], st["eta"], st["U"], st["W"])
    out = torch.empty((3, 8), dtype=torch.float64, device="cuda")
    try:
        for _ in range(2):
            ens.step(2)
            ref = ens.stats(0)                      # existing entry point (synchronises)
            with torch.cuda.stream(ens.stream):
                out.fill_(float("nan"))             # every value must be written by the call
            dns.dns_stats_noalloc(ens.h, 0, out.data_ptr())
            ens.stream.synchronize()
            got = out.cpu().numpy()
            for i, k in enumerate(KEYS):
                want = np.asarray(ref[k], dtype=np.float64)
                if k == "max_div":
                    assert np.all(np.abs(got[:, i] - want) <= 1e-13), k
                else:
                    assert np.all(np.abs(got[:, i] - want) <= 1e-12 * max(1.0, np.abs(want).max())), k
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
