"""Compile the CPU oracle (test infrastructure) with gcc.

oracle/liboracle.so: the lexicographic oracle (mg_oracle.c), single-threaded.
oracle/liboracle_colour.so: the four-colour OpenMP baseline (mg_oracle_colour.c,
which includes mg_oracle.c).
FP contraction is switched off so that x86-64 and aarch64 hosts round alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mg_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")
SRC_COLOUR = os.path.join(HERE, "mg_oracle_colour.c")
OUT_COLOUR = os.path.join(HERE, "liboracle_colour.so")

_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-Wextra",
          "-Wno-unused-parameter"]


def _stale(out, srcs):
    return not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out)
                                          for s in srcs)


def build(force: bool = False) -> str:
    if force or _stale(OUT, [SRC]):
        subprocess.run(["gcc"] + _FLAGS + ["-o", OUT, SRC, "-lm"], check=True)
    return OUT


def build_colour(force: bool = False) -> str:
    if force or _stale(OUT_COLOUR, [SRC, SRC_COLOUR]):
        subprocess.run(["gcc"] + _FLAGS + ["-fopenmp", "-o", OUT_COLOUR, SRC_COLOUR, "-lm"],
                       check=True)
    return OUT_COLOUR


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_colour(force="--force" in sys.argv))
