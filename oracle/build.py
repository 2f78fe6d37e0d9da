"""Compile the CPU oracle (test infrastructure only) into oracle/_build/liboracle.so.

Plain gcc, no CUDA: the oracle shares nothing with the GPU library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "qubo_oracle.c"), os.path.join(HERE, "qubo_oracle_blocked.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and all(
            os.path.getmtime(LIB) >= os.path.getmtime(src) for src in SRCS):
        return LIB
    cmd = [
        os.environ.get("CC", "gcc"), "-O3", "-std=c11", "-fPIC", "-shared",
        "-ffp-contract=off", "-fno-fast-math", "-pthread", "-Wno-psabi",
        *SRCS, "-o", LIB + ".tmp", "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
