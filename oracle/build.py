"""Compile the CPU oracle (oracle.c) into oracle/liboracle.so with the host C compiler.

Test infrastructure only: the oracle is built so that the tests, the smoke check
and the benchmark's CPU-baseline leg can call it; the CUDA library never does.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def compile_to(src: str, out: str) -> str:
    """Compile one C source with the oracle's flags into the shared library `out`."""
    cc = os.environ.get("CC", "gcc")
    # -ffp-contract=off: every product and sum is rounded on its own, as written.
    cmd = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", out + ".tmp", src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    return compile_to(SRC, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
