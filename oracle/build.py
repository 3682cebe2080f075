"""Compile the oracle's C source with gcc into oracle/_build/liborc.so.

Building the checker is not using it: ``__graft_entry__.build()`` calls this
so that the tests find the library on any machine (x86 here, aarch64 on the
GPU host).  Portable C only: no -march flags, no intrinsics.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "liborc.so")


def build_oracle(force: bool = False) -> str:
    out = library_path()
    src = os.path.join(_HERE, "orc.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
