"""Compile the C oracle (test infrastructure only) into oracle/libjl_oracle.so.

Flags: -O2 -ffp-contract=off and no fast-math, so each C statement of the
iteration is one correctly rounded IEEE operation (no fused multiply-add) and
subnormals are kept.  Run as ``python oracle/build.py``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jl_oracle.c")              # Z^2 + C (Sec. 2, 3)
MAPS_SRC = os.path.join(HERE, "jl_oracle_maps.c")    # Z^d + C and P/Q + C (Sec. 2, Fig. 4)
MAPS_INC = os.path.join(HERE, "map_iter.inc")
LIB = os.path.join(HERE, "libjl_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-fno-finite-math-only", "-frounding-math", "-pthread"]


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(f) for f in (SRC, MAPS_SRC, MAPS_INC))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, "-I", HERE, SRC, MAPS_SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
