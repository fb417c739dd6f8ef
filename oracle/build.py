"""Compile the C oracle into ``oracle/_liboracle.so`` with gcc.

Test infrastructure: building the checker is not using it; ``build()`` of the
package compiles it alongside the CUDA library so the tests find it ready.
Flags keep FP64 semantics identical on x86_64 and aarch64: no fast-math and
no contraction of a*b+c into fused multiply-adds.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mact_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")


def compile_lib(src: str, out: str) -> str:
    """gcc one oracle source into a shared library at out (atomically)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    return compile_lib(SRC, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
