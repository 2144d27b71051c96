"""Builds libapsp.so (the C-ABI CUDA library) in-tree for sm_103a.

    python -m paper_1001_4108_gb300.build [--force] [--verbose]

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into paper_1001_4108_gb300/_lib/libapsp.so with the CUDA
runtime linked statically (the library then works next to any PyTorch build).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libapsp.so")
SOURCES = ["api.cu", "fw_i32.cu", "fw_f32.cu", "fw_i16.cu", "ubench.cu", "noalloc.cu", "batched.cu", "tuning.cu", "server.cu",
           "paths.cu", "selftest.cu", "checks.cu", "dataflow.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libapsp")


def _deps(src: str):
    yield os.path.join(CSRC, src)
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h")):
            yield os.path.join(CSRC, f)
    yield os.path.join(ROOT, "include", "apsp.h")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False,
          defines=(), out_dir: str | None = None) -> str:
    """Compile and link libapsp.so; returns its path.  ``defines`` (e.g.
    ["APSP_P3_MINB=1"]) and ``out_dir`` build a tuning variant elsewhere."""
    nvcc = _nvcc()
    out_dir_ = OUT_DIR if out_dir is None else out_dir
    obj_dir = OBJ_DIR if out_dir is None else os.path.join(out_dir, "_build")
    lib = os.path.join(out_dir_, "libapsp.so")
    os.makedirs(out_dir_, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    dflags = [f"-D{d}" for d in defines]
    jobs = []
    for src in SOURCES:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        if force or _stale(obj, list(_deps(src))):
            cmd = [nvcc] + NVCC_FLAGS + dflags + (["-Xptxas", "-v"] if ptxas_verbose else []) + \
                  ["-c", os.path.join(CSRC, src), "-o", obj]
            jobs.append((src, cmd))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src for src, cmd in jobs}
            failed = []
            for f in cf.as_completed(futs):
                r = f.result()
                if verbose or ptxas_verbose or r.returncode:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode:
                    failed.append(futs[f])
            if failed:
                raise RuntimeError(f"nvcc failed for {failed}")
    objs = [os.path.join(obj_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print ptxas register/smem usage")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, ptxas_verbose=a.ptxas))
