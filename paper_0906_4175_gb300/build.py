"""Build libmfgb.so in-tree with nvcc for sm_103a (one -gencode, parallel TUs).

    python -m paper_0906_4175_gb300.build [--verbose] [--force] [--debug]

Output: paper_0906_4175_gb300/_build/libmfgb.so (git-ignored); --debug builds
the index-checking variant (-DMFGB_DEBUG, see mf_debug_status) into _build_debug/.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libmfgb.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
SOURCES = ["mf_filter.cu", "mf_persist.cu", "mf_prep.cu", "mf_synth.cu", "mf_refine.cu", "mf_chisq.cu", "mf_events.cu", "mf_rows.cu", "mf_pass1.cu", "mf_prep64.cu", "mf_fused.cu", "mf_api.cu"]
HEADERS = ["mf_fft.cuh", "mf_passes.cuh", "mf_filter.cuh", "mf_internal.h", "mf_tmpl.cuh", "mf_async.cuh", "mf_pass1.cuh", "mf_rows.cuh"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    return "/usr/local/cuda"


def nvcc_flags(verbose: bool = False, debug: bool = False):
    f = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if debug:
        f += ["-DMFGB_DEBUG"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "mfgb.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every CUDA translation unit and link libmfgb.so; returns its path."""
    out_dir = BUILD_DEBUG if debug else BUILD
    lib = os.path.join(out_dir, "libmfgb.so")
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = os.path.join(_cuda_home(), "bin", "nvcc")
    flags = nvcc_flags(verbose, debug)

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for src, _, r in results:
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-cudart", "shared",
           "-Xlinker", "-rpath," + os.path.join(_cuda_home(), "lib64"), "-o", tmp] + [o for _, o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
