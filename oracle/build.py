"""Compile the C oracle into oracle/_build/liblbm_wenoc_oracle.so with gcc.

Test infrastructure: building the checker is not using it.  Plain C99, no
architecture flags (the same source builds on x86_64 and aarch64), FMA
contraction off so the result does not depend on the host's instruction set.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_wenoc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_wenoc_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # -fcx-limited-range: plain complex division in the reverse sweep's complex-step twins
    # (the forward uses no complex arithmetic)
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fcx-limited-range",
           "-fopenmp", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
