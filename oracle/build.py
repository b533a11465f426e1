"""Compile the FP64 C oracle into oracle/_build/liboracle.so (test infrastructure)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sssgs_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


# -ffp-contract=off: the float32 depth key uses explicit fmaf only.
FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def compile_library(src: str, out: str) -> None:
    """gcc: C source -> shared library, with the oracle's flags."""
    subprocess.run(["gcc", *FLAGS, src, "-o", out, "-lm"], check=True)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    tmp = OUT + f".{os.getpid()}.tmp"
    compile_library(SRC, tmp)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
