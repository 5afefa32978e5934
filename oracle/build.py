"""Build the CPU oracle (test infrastructure only) into oracle/liboracle.so.

Compiled with -ffp-contract=off so that the encoding FFT performs exactly the
IEEE-754 products and sums its source states (no fused multiply-add).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    src = [os.path.join(HERE, "oracle.c")]
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(f) for f in src + [hdr, __file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", LIB + ".tmp"] + src + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
