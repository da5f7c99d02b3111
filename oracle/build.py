"""Build the FP64 CPU oracle (test infrastructure only).

Compiles ``lbd_oracle.c`` into ``liborc.so`` (2D) and ``lbd_oracle3.c`` into
``liborc3.so`` (3D) beside this file with plain gcc,
``-O2 -ffp-contract=off`` (no fused multiply-adds, so the arithmetic is the IEEE
sequence written in the source) and OpenMP for the row loops.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbd_oracle.c")
LIB = os.path.join(HERE, "liborc.so")
SRC3 = os.path.join(HERE, "lbd_oracle3.c")
LIB3 = os.path.join(HERE, "liborc3.so")


def _compile(src, lib, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Build both oracles; returns the path of the 2D one."""
    _compile(SRC3, LIB3, force)
    return _compile(SRC, LIB, force)


def build3(force: bool = False) -> str:
    return _compile(SRC3, LIB3, force)


if __name__ == "__main__":
    print(build(force=True))
