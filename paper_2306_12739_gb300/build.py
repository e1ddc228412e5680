"""Build libdns.so in-tree for sm_103a (nvcc + g++, no cmake).

The translation units compile in parallel; the shared library lands next to
this file as ``libdns.so``.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdns.so")
# the bounds-checked debug build (-DDNS_CHECK), loaded when DNS_CHECKED=1
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libdns_check.so")
ROOT = os.path.dirname(HERE)

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
           "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + os.path.join(ROOT, "include")]

CU = ["api.cu", "k_spectral.cu", "k_plane.cu", "k_plane_f32.cu", "k_gemm_f32.cu", "k_noalloc.cu", "k_yderiv_tc.cu", "k_plane_cl.cu", "k_plane_lines.cu", "k_helm_tc.cu", "k_linear.cu", "k_stoch.cu", "k_spec.cu", "k_d2v_tc.cu", "k_step_eo.cu"]
CPP = ["builder.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP]


def _deps():
    return _sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                         if f.endswith((".hpp", ".cuh", ".h"))] + [os.path.join(ROOT, "include", "dns.h")]


def _compile(src, extra=(), build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        cmd = [NVCC] + ARCH + NVFLAGS + list(extra) + ["-c", src, "-o", obj]
    else:
        cmd = ["g++"] + CXXFLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def _locked(fn):
    """Serialise concurrent builds (several ranks on one node) with a file lock."""
    def wrap(*a, **k):
        import fcntl
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), ".build.lock"), "w") as lk:
            fcntl.flock(lk, fcntl.LOCK_EX)
            try:
                return fn(*a, **k)
            finally:
                fcntl.flock(lk, fcntl.LOCK_UN)
    return wrap


@_locked
def build(force=False, verbose=False, extra_nvcc=(), checked=False):
    """Build libdns.so (or, with checked, the bounds-checked libdns_check.so)."""
    lib, bdir = (LIB_CHECK, BUILD_CHECK) if checked else (LIB, BUILD)
    extra = tuple(extra_nvcc) + (("-DDNS_CHECK",) if checked else ())
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in _deps())):
        return lib
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(_sources())) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, bdir), _sources()))
    if verbose:
        for _, err in results:
            if err:
                print(err)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra_nvcc=sys.argv[1:]))
