"""Compile the FP64 oracle (plain C) into oracle/_build/liboracle.so, and the same source narrowed
to single precision (oracle_f32.c) into oracle/_build/liboracle_f32.so.

Test infrastructure: built with gcc, no vectorisation flags, FMA contraction off so
that x86-64 and aarch64 hosts produce the same doubles.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB32 = os.path.join(OUT_DIR, "liboracle_f32.so")
SRC = os.path.join(HERE, "oracle.c")
SRC32 = os.path.join(HERE, "oracle_f32.c")


def _compile(src, lib, deps, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Both builds; returns the FP64 library's path."""
    _compile(SRC32, LIB32, (SRC, SRC32), force)
    return _compile(SRC, LIB, (SRC,), force)


def build_f32(force: bool = False) -> str:
    build(force)
    return LIB32


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
