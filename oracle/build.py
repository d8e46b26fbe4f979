"""Build step for the oracle (test infrastructure only).

Compiles ``adpar_oracle.c`` with gcc into ``liboracle.so`` beside it.  The
flags keep FP64 semantics plain: no fast-math and no contraction of a*b+c
into a fused multiply-add, so the x86 and Arm builds round identically.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "adpar_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build_oracle(force=False):
    """Compile the oracle shared library if it is missing or stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
