"""Compiles the oracle's C sources into oracle/_oracle.so (gcc, OpenMP, FP64).

Test infrastructure only: the product library never loads the result.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["hfmm_oracle.c", "hfmm_oracle_fmm.c"]
TARGET = os.path.join(HERE, "_oracle.so")


def needs_build() -> bool:
    if not os.path.exists(TARGET):
        return True
    t = os.path.getmtime(TARGET)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES)


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = TARGET + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off",  # same rounding on x86-64 and aarch64
            *[os.path.join(HERE, s) for s in SOURCES], "-lm", "-o", tmp,
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force=True))
