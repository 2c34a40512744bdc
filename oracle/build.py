"""Compile the C oracle into ``oracle/_build/libd2q9_oracle.so`` with gcc.

The oracle is test infrastructure (see ``oracle/__init__.py``). Flags keep the
arithmetic the same on x86_64 and aarch64: no FMA contraction, no fast-math.
With OpenMP the sweeps can run on several threads (``d2q9.set_threads``).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "d2q9_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libd2q9_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-Wall", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    # OpenMP for the multi-threaded timing of the sweeps; without it the
    # oracle is built serial (oracle_openmp() then reports 0)
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
