"""Register and local-memory budgets of the hot-path kernels, from ptxas's own
report (-Xptxas -v) of the sm_103a build: the occupancy the design relies on
(three CTAs per SM for the fused stage in parity blocks, one 800-thread CTA per
SM for the 64-point plane stage) and no spills in the kernels that run every
sub-step.  CPU only: nvcc cross-compiles."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_12739_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

# translation units of the hot path, and the kernels in them that must not spill
UNITS = ["k_spec.cu", "k_step_eo.cu", "k_plane_lines.cu", "k_yderiv_tc.cu", "k_d2v_tc.cu"]
NO_SPILL = ("k_spec_eo", "k_eo_derivs", "k_spec", "k_plane_lines", "k_yderiv_eo", "k_forcing_eo", "k_helm_eo",
            "k_yderiv_tc", "k_d2v_tc")


def _report(unit, tmp):
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"),
           "-Xptxas", "-v", "-c", os.path.join(CSRC, unit), "-o", os.path.join(tmp, unit + ".o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, cur = {}, None
    for ln in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", ln)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", ln)
        if m and cur:
            out.setdefault(cur, {})["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", ln)
        if m and cur:
            out.setdefault(cur, {})["regs"] = int(m.group(1))
            cur = None
    return out


@pytest.fixture(scope="module")
def reports(tmp_path_factory):
    if not (os.path.exists(NVCC) or shutil.which("nvcc")):
        pytest.skip("no nvcc")
    tmp = str(tmp_path_factory.mktemp("ptxas"))
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        parts = list(ex.map(lambda u: _report(u, tmp), UNITS))
    rep = {}
    for p in parts:
        rep.update(p)
    return rep


def test_hot_kernels_do_not_spill(reports):
    seen = set()
    for mangled, r in reports.items():
        for k in NO_SPILL:
            if re.search(r"\d" + k + r"(?:I|E)", mangled):
                seen.add(k)
                assert r.get("spill", 0) == 0, (mangled, r)
    assert seen == set(NO_SPILL), sorted(set(NO_SPILL) - seen)


def test_register_budgets_the_occupancy_relies_on(reports):
    def regs(pattern):
        hits = [r["regs"] for m, r in reports.items() if re.search(pattern, m)]
        assert hits, pattern
        return max(hits)
    # the fused stage in parity blocks at three CTAs per SM: 3 x 256 threads x 80 registers
    assert regs(r"k_spec_eoILi63ELi4ELi3ELb1E") <= 80
    # the 64-point plane stage: one CTA of 800 threads per SM
    assert regs(r"k_plane_linesILi64ELi64ELb0E") * 800 <= 65536
    # the parity-block apply at three CTAs of 256 threads per SM
    assert regs(r"k_helm_eo") * 256 * 3 <= 65536
