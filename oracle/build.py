"""Compile the C oracle into ``oracle/liborc.so``.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library and is never
called by it.  Building it is a plain gcc call (no CUDA), so it works on the
x86 container and on the Arm GPU host alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("clbm_oracle.c", "clbm_oracle3d.c")]
HDRS = [os.path.join(HERE, f) for f in ("clbm_oracle.h", "clbm_oracle3d.h")]
LIB = os.path.join(HERE, "liborc.so")


def build(force: bool = False) -> str:
    """Build liborc.so if it is missing or older than its sources; return its path."""
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(p) for p in SRCS + HDRS)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared"] + SRCS + ["-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
