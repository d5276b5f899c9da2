"""In-tree build of libfem.so for sm_103a with nvcc (no cmake, no torch
extension machinery).  Every .cu/.cpp file under csrc/ is compiled to an
object in parallel, then linked into paper_2204_03893_gb300/libfem.so."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfem.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "fem.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    hmt = _headers_mtime()
    objs, todo = [], []
    for src in _sources():
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(sp), hmt):
            cmd = [nv, *ARCH, *FLAGS, "-c", sp, "-o", obj]
            if ptxas_verbose and src.endswith(".cu"):
                cmd[1:1] = ["-Xptxas", "-v"]
            todo.append((src, cmd))

    def run(item):
        src, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    jobs = jobs or min(8, os.cpu_count() or 4)
    errors = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for src, r in ex.map(run, todo):
            if verbose or r.returncode != 0 or ptxas_verbose:
                sys.stderr.write(f"--- {src}\n{r.stdout}{r.stderr}")
            if r.returncode != 0:
                errors.append(src)
    if errors:
        raise RuntimeError(f"nvcc failed for {errors}")
    if todo or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv)
    print(LIB)
