"""Build the bp_gb300 shared library for sm_103a with nvcc (in-tree).

Each .cu file compiles in parallel to an object, then one link step makes
paper_2401_09283_gb300/_build/libbp_gb300.so.  Only the GB300 target is
built: -gencode arch=compute_103a,code=sm_103a.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbp_gb300.so")
SOURCES = ["bp_api.cu", "bp_job.cu", "bp_geom.cu", "bp_project.cu", "bp_noalloc.cu", "bp_spline.cu",
           "bp_fdk.cu", "bp_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build bp_gb300")
    return cand


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra)


# Variants: the release library, and a debug library with every gather and
# scatter index checked (-DBP_BOUNDS_CHECK; bp_bounds_check reports failures).
VARIANTS = {"release": (BUILD, LIB, []),
            "bounds": (os.path.join(HERE, "_build_bc"),
                       os.path.join(HERE, "_build_bc", "libbp_gb300_bc.so"),
                       ["-DBP_BOUNDS_CHECK"])}


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "bp_gb300.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False, extra=(), variant="release") -> str:
    build_dir, lib, vflags = VARIANTS[variant]
    if not force and not _stale(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(list(vflags) + list(extra))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared"] + ARCH + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose="-v" in sys.argv,
                        extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
