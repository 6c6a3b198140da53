"""Builds libttie.so (CUDA, sm_103a) in-tree with nvcc: one object per translation
unit, compiled in parallel, then linked into a shared library beside this file."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libttie.so")
UNITS = ["sort_scan.cu", "bvh.cu", "hash.cu", "pair_eval.cu", "assemble.cu", "pcg.cu", "instances.cu", "capi.cu", "pcg_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


LIB_CHECKED = os.path.join(HERE, "libttie_checked.so")


def flags(extra=(), checks=None):
    # TTIE_BUILD_CHECKS=1 builds the self-checking variant (bounds checks, a sync after every launch)
    if checks is None:
        checks = os.environ.get("TTIE_BUILD_CHECKS") == "1"
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                   "-I", SRC] + (["-DTTIE_CHECKS"] if checks else []) + list(extra)


def _stamp():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(ROOT, "include", "ttie.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    """Builds libttie.so (or, with checked, the self-checking libttie_checked.so beside it,
    leaving libttie.so as it is) and returns its path."""
    lib = LIB_CHECKED if checked else LIB
    out_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    force = force or (not checked and os.environ.get("TTIE_BUILD_CHECKS") == "1")
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _stamp() and not ptxas_info:
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_unit(u):
        obj = os.path.join(out_dir, u.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(SRC, u), "-o", obj] + flags(extra, True if checked else None)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (u, r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        res = list(ex.map(compile_unit, UNITS))
    if verbose or ptxas_info:
        for _, err in res:
            sys.stderr.write(err)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in res] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
