"""Build libhfv.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit compiles in parallel; the shared library lands next to
this file.  Nothing here needs a GPU: nvcc cross-compiles.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhfv.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["mesh.cpp", "scheme.cpp", "setup.cu", "residual.cu", "residual_2d.cu", "residual_2d_high.cu", "residual_3d.cu",
         "residual_hex.cu", "residual_hex5.cu", "residual_hex6.cu", "adjoint.cu", "api.cu", "noalloc.cu", "peak.cu"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "hfv.h"))
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "--expt-relaxed-constexpr"] + ARCH + (extra or [])
    jobs = []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(BUILD, u + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            if u.endswith(".cpp"):
                cmd = [nvcc, "-x", "cu"] + flags + ["-c", src, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for log in ex.map(run, jobs):
            if verbose and log.strip():
                print(log)
    objs = [os.path.join(BUILD, u + ".o") for u in UNITS]
    if force or jobs or not os.path.exists(OUT):
        tmp = OUT + f".{os.getpid()}.tmp"
        run([nvcc, "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcudart", "-lpthread"])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
