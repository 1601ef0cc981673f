"""Compile the CPU oracle (``fv_oracle.c``, ``mlp_oracle.c``) into ``oracle/_build/liboracle.so``.

Test infrastructure: the oracle is built with ``-ffp-contract=off`` so that no
multiply-add is fused behind the source's back (on aarch64 GCC fuses by
default), and with OpenMP when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "fv_oracle.c"), os.path.join(HERE, "mlp_oracle.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def compile_lib(srcs, out: str, verbose: bool = False) -> str:
    """Compile C sources into the shared library ``out`` with the oracle's
    flags (OpenMP when the compiler has it)."""
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            *srcs, "-o", out + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode == 0:
            os.replace(out + ".tmp", out)
            return out
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in SRCS)):
        return LIB
    return compile_lib(SRCS, LIB, verbose)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
