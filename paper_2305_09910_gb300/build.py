"""Builds liblbm.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

The library is compiled from ``csrc/``: one host/API translation unit plus one kernel
translation unit per (stencil, storage precision) pair, compiled in parallel and linked
with the static CUDA runtime.  A hash of the sources and flags is stored next to the
library so an unchanged tree is not rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liblbm.so")
BUILD = os.path.join(PKG, "_build")
# variants: "check" = every global access of the direct kernels bounds-checked (a checked
# access outside its array is skipped and reported by lbm_sync), for memory-safety tests
VARIANTS = {None: ("liblbm.so", "_build", []), "check": ("liblbm_check.so", "_build_check", ["-DLBM_BOUNDS_CHECK"])}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

INSTANCES = [(q, s) for q in (19, 27) for s in ("float", "__half", "__nv_bfloat16")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh", ".h"))) + [os.path.join(INCLUDE, "lbm.h")]


def _digest(extra) -> str:
    h = hashlib.sha256()
    for path in _sources():  # paths relative to the repository: the same stamp on every machine
        with open(path, "rb") as fh:
            h.update(os.path.relpath(path, ROOT).encode() + b"\0" + fh.read())
    flags = " ".join(ARCH + NVFLAGS + list(extra)).replace(ROOT, ".")  # no machine paths
    h.update(flags.encode())
    return h.hexdigest()


def _kernel_sources():
    """The sources of the step-kernel translation units (kern_inst.cu and the headers it includes)."""
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")) + \
        [os.path.join(CSRC, "kern_inst.cu")]


def _code_only(text: str) -> str:
    """The source without its comments, trailing blanks and empty lines (the kernel sources hold
    no comment markers inside string literals)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_digest(extra=()) -> str:
    """Hash of the step kernels' code (comments excluded) and flags: ncu summaries taken on one
    build stay valid for another with the same kernels (host-side API changes and comment edits
    do not touch them)."""
    h = hashlib.sha256()
    for path in _kernel_sources():
        with open(path, encoding="utf-8") as fh:
            h.update(os.path.relpath(path, ROOT).encode() + b"\0" + _code_only(fh.read()).encode())
    h.update(" ".join(ARCH + NVFLAGS + list(extra)).replace(ROOT, ".").encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant=None) -> str:
    """Compiles (if needed) and returns the path of liblbm.so (or of a variant's library)."""
    name, bdir, vflags = VARIANTS[variant]
    lib_path = os.path.join(PKG, name)
    build_dir = os.path.join(PKG, bdir)
    extra = list(vflags) + list(extra_flags)
    digest = _digest(extra)
    stamp = lib_path + ".sha256"
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                with open(lib_path + ".kernel.sha256", "w") as kfh:
                    kfh.write(kernel_digest(extra) + "\n")
                return lib_path
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    jobs = [(os.path.join(CSRC, "lbm_api.cu"), os.path.join(build_dir, "lbm_api.o"), []),
            (os.path.join(CSRC, "lbm_noalloc.cu"), os.path.join(build_dir, "lbm_noalloc.o"), []),
            (os.path.join(CSRC, "lbm_closure.cu"), os.path.join(build_dir, "lbm_closure.o"), [])]
    for q, s in INSTANCES:
        tag = s.strip("_").replace("nv_", "")
        jobs.append((os.path.join(CSRC, "kern_inst.cu"), os.path.join(build_dir, f"kern_q{q}_{tag}.o"),
                     [f"-DLBM_Q={q}", f"-DLBM_S={s}"]))

    def compile_one(job):
        src, obj, defs = job
        cmd = [nvcc, *ARCH, *NVFLAGS, *extra, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(compile_one, jobs))
    if verbose:
        for log in logs:
            if log:
                sys.stderr.write(log)
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + [j[1] for j in jobs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {name} failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(digest + "\n")
    with open(lib_path + ".kernel.sha256", "w") as fh:
        fh.write(kernel_digest(extra) + "\n")
    return lib_path


if __name__ == "__main__":
    v = "-v" in sys.argv
    flags = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force="--force" in sys.argv, verbose=v or bool(flags), extra_flags=flags))
