"""Builds libemb.so in-tree: every csrc/*.cu compiled for sm_103a in parallel, then linked.

Usage: python -m paper_2512_01251_gb300.build [--force] [--verbose-ptxas] [--check]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libemb.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(HERE, "..", "include", "emb.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


CHECK_LIB = os.path.join(OUT_DIR, "libemb_check.so")


def build(force: bool = False, ptxas_verbose: bool = False, check: bool = False) -> str:
    """Compile and link libemb.so; returns its path.  Raises on compiler errors.
    check=True builds libemb_check.so instead: the same library with the bounds mode
    (-DEMB_CHECK) that turns an out-of-range index into the device status
    EMB_ERR_BOUNDS."""
    out_dir = os.path.join(OUT_DIR, "check") if check else OUT_DIR
    lib = CHECK_LIB if check else LIB
    os.makedirs(out_dir, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs = []
    procs = []
    for src in srcs:
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [NVCC, *ARCH, *FLAGS, *(["-DEMB_CHECK"] if check else []), "-c", src, "-o", obj + ".tmp"]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, obj, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"--- {os.path.basename(src)}\n{out.decode(errors='replace')}")
        else:
            os.replace(obj + ".tmp", obj)
            if ptxas_verbose and out:
                sys.stdout.write(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    if force or procs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, ptxas_verbose="--verbose-ptxas" in sys.argv, check="--check" in sys.argv))
