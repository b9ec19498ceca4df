"""Build libvms_gb300.so for sm_103a with nvcc (translation units compiled in parallel).

Usage: python -m paper_0809_4802_gb300.build [--verbose] [--ptxas-info]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvms_gb300.so")
SOURCES = ["api.cu", "residual.cu", "tangent.cu", "misc.cu", "solver.cu", "pattern.cpp", "ts_plan.cpp", "band_order.cpp", "noalloc.cu", "precond.cu", "mlp.cu", "tet.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(src: str, ptxas_info: bool) -> list[str]:
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include")]
    if src.endswith(".cu"):
        f = ARCH + common + ["-lineinfo", "--expt-relaxed-constexpr"]
        if ptxas_info:
            f += ["-Xptxas", "-v"]
        return f
    return common + ["-x", "c++"]


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "vms.h"))
    newest_header = max(os.path.getmtime(h) for h in headers)

    def compile_one(src: str):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        if (not force and not ptxas_info and os.path.exists(o)
                and os.path.getmtime(o) >= max(os.path.getmtime(s), newest_header)):
            return o, ""
        cmd = [cc] + _flags(src, ptxas_info) + ["-c", s, "-o", o]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
        return o, p.stdout + p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for _, log in results:
        if log and (verbose or ptxas_info):
            print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(a.verbose, a.ptxas_info, a.force))
