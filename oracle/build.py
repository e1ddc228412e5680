"""Compile the oracle's quad-precision operator builder (test infrastructure only).

Produces ``oracle/liboracle_ops.so`` next to this file.  Plain gcc, no CUDA.
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ops_quad.c")
LIB = os.path.join(HERE, "liboracle_ops.so")


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
def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           SRC, "-o", LIB + ".tmp"]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    cmd.append("-lm")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
