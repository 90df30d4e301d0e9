"""Build the oracle shared library (test infrastructure only).

The oracle is compiled with IEEE-754 semantics and no fused multiply-add,
so that every binary32/binary64 operation in ssa_oracle.c is one correctly
rounded operation on any host (x86_64 or aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssa_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
FLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fno-strict-aliasing",
         "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *FLAGS, SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
