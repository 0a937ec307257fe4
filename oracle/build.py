"""Compile the oracle's C source into ``oracle/_build/liboracle.so`` (serial) and
``oracle/_build/liboracle_omp.so`` (the same source with OpenMP: cell loops and
per-particle updates on all cores, bitwise identical results).

The oracle is test infrastructure (see ``pibm_oracle.c``). It is compiled with
FP contraction off so that every operation rounds as written, on x86_64 and
aarch64 alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pibm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _compile(out, extra):
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *extra, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, parallel: bool = False) -> str:
    """Path of the serial library (parallel=False) or of the OpenMP one."""
    os.makedirs(OUT_DIR, exist_ok=True)
    out = LIB_OMP if parallel else LIB
    if force and os.path.exists(out):
        os.remove(out)
    return _compile(out, ["-fopenmp"] if parallel else [])


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, parallel=True))
