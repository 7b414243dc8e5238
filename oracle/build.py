"""Compile the oracle's C routines (test infrastructure only).

The oracle is a plain FP64 CPU implementation used by tests/, by
``__graft_entry__.smoke()`` and by bench.py's CPU-baseline leg. Building it
does not make the library depend on it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "evx_oracle.c")
LIB = os.path.join(HERE, "liborc.so")


def build_oracle(force: bool = False) -> str:
    """Build ``oracle/liborc.so`` with gcc + OpenMP if missing or stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
