"""Build the C part of the FP64 oracle (test infrastructure only).

Compiles ``krr_oracle.c`` into ``_liboracle.so`` beside it with plain gcc:
``-O2 -fopenmp -ffp-contract=off`` (no fused multiply-add contraction and no
fast-math, so the arithmetic is the C source's own, on x86 and Arm alike).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "krr_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
