"""Build libctfmnmf.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
``paper_2510_02382_gb300/_build/libctfmnmf.so`` (git-ignored). Run as
``python -m paper_2510_02382_gb300.build`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB_NAME = "libctfmnmf.so"
SOURCES = ["api.cpp", "batch_api.cpp", "kernels.cu", "bin_phase.cu", "batch.cu", "persistent.cu", "noalloc.cu", "grad.cu", "grad_api.cpp", "cluster_bin.cu"] + [f"{k}_m{m}.cu" for k in ("persistent", "bin_phase", "batch")
                                                         for m in range(2, 9)] + [f"grad_bin_m{m}.cu" for m in range(2, 5)] \
    + [f"bin_contig_m{m}.cu" for m in range(2, 5)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


DEBUG_DIR = os.path.join(PKG, "_build_debug")


def lib_path(debug: bool = False) -> str:
    """The release library, or (debug) the CTFMNMF_DEBUG build with device bounds checks and a
    NaN/Inf scan after every iteration."""
    return os.path.join(DEBUG_DIR if debug else OUT_DIR, LIB_NAME)


def is_stale() -> bool:
    """True if the library is missing or older than any of its sources or headers."""
    if not os.path.exists(lib_path()):
        return True
    t = os.path.getmtime(lib_path())
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    return any(os.path.getmtime(p) > t for p in deps)


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), *extra]


def build(verbose: bool = False, ptxas_verbose: bool = False, debug: bool = False) -> str:
    out_dir = DEBUG_DIR if debug else OUT_DIR
    os.makedirs(out_dir, exist_ok=True)
    nvcc = nvcc_path()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    if debug:
        extra.append("-DCTFMNMF_DEBUG")

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd += ["-x", "cu"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        return obj, res.stdout + res.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    logs = "".join(r[1] for r in results)
    tmp = lib_path(debug) + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[r[0] for r in results]]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path(debug))
    if verbose or ptxas_verbose:
        sys.stdout.write(logs)
    return lib_path(debug)


if __name__ == "__main__":
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv, debug="--debug" in sys.argv))
