"""Compile the C oracle into oracle/liboracle.so (gcc, -O2, OpenMP).

The oracle is plain C with no BLAS; this script only builds the checker.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "gpbo_oracle.c"), os.path.join(HERE, "mlp_oracle.c"), os.path.join(HERE, "mle_oracle.c")]
OUT = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [s for s in SRC if os.path.exists(s)]
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return OUT
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-o", OUT] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
