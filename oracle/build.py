"""Compile the FP64 CPU oracle into oracle/_build/liborc.so.

TEST INFRASTRUCTURE ONLY: the oracle is the reference the CUDA path is checked
against; nothing on the product path links or loads it.

Flags: -O2 and -ffp-contract=off so that no multiply-add is fused and every
rounding is the one written in the source (aarch64 compilers fuse by default);
-fopenmp for the loops over blocks and cells that the timed CPU baseline runs on
all host cores (orc_set_threads; every such loop gives the serial result).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["euler.cpp", "exact_riemann.cpp", "mg.cpp", "amg.cpp", "cnn.cpp"]
OUT = os.path.join(HERE, "_build", "liborc.so")


def build(force: bool = False, extra_flags: list[str] | None = None, out: str = OUT) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    deps = srcs + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(out):
        mt = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= mt for d in deps) and not extra_flags:
            return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", out + ".tmp"] + (extra_flags or []) + srcs
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
