"""Build the CPU oracle shared library (test infrastructure only).

The oracle is compiled with ``-O2 -ffp-contract=off -fno-fast-math`` so that each
floating-point operation in ``jacobi_oracle.c`` is one IEEE-754 round-to-nearest
operation in source order, and with OpenMP for the optional loop over k (which
does not change any result).  No architecture-specific flags are used, so the
same source gives the same bits on x86-64 (SSE2) and AArch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jacobi_oracle.c")
LIB = os.path.join(HERE, "libjacobi_oracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=c11", "-fopenmp", "-Wall", "-Wno-unknown-pragmas"]


def build(src: str = SRC, out: str = LIB, extra=()) -> str:
    """Compile ``src`` into the shared library ``out`` unless it is up to date."""
    if (os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)
            and not extra):
        return out
    cmd = ["gcc", *CFLAGS, *extra, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(*sys.argv[1:]))
