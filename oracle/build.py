"""Build step for the CPU oracle (test infrastructure only).

Compiles ``ugkwp_oracle.c`` (the step) and ``ugkwp_oracle_tangent.c`` (its
pathwise derivative) with gcc into ``liboracle.so`` beside them.
``-ffp-contract=off`` keeps the arithmetic identical on x86-64 and AArch64
(no fused multiply-adds are formed on either).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("ugkwp_oracle.c", "ugkwp_oracle_tangent.c")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        [os.path.getmtime(s) for s in SRCS] + [os.path.getmtime(os.path.join(HERE, "ugkwp_oracle.h"))]
    ):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", *SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
