"""Compile the C oracle (oracle.c) into oracle/liboracle.so with the host C compiler.

The oracle is test infrastructure: this step only builds the checker, it never runs it.
OpenMP is used when the compiler supports it; the oracle is correct either way.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))
    ):
        return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), r.stdout, r.stderr, file=sys.stderr)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError(f"oracle build failed:\n{r.stderr}")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
