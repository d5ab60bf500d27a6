"""Compile the FP64 CPU oracle (plain C) into ``oracle/liboracle_fdm.so``.

Test infrastructure only: building the checker is not using it.  No optimisation
flag changes the arithmetic (``-ffp-contract=off`` keeps x86-64 and AArch64 results
bit-identical; no fast-math).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fdm_oracle.c")
LIB = os.path.join(HERE, "liboracle_fdm.so")


def build_oracle(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, SRC, "-lm"]
    # OpenMP splits the loops over independent rows and nodes across threads (results do
    # not depend on the thread count); without it the library is the serial program
    if subprocess.call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
