"""Build the serial C oracle into ``oracle/liboracle.so``.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark load this library; the product library never does.

Flags: ``-O2 -fwrapv -ffp-contract=off`` and no fast-math, so integer
arithmetic wraps and the float program rounds after every multiply and add, as
the serial C program of the region does (IPMACC Sec. 1.3, Listing 1a).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
CFLAGS = ["-std=c99", "-O2", "-fwrapv", "-ffp-contract=off", "-fno-fast-math",
          "-Wall", "-Wextra", "-fPIC", "-shared"]


def build(force=False):
    """Compile the oracle if the shared library is missing or stale."""
    hdr = os.path.join(HERE, "oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [os.environ.get("CC", "gcc")] + CFLAGS + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
