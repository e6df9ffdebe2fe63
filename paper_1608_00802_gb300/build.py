"""Builds libpm.so (the C-ABI library) in-tree for sm_103a with nvcc.

The translation units compile in parallel (host API, fp32 kernels, fp64
kernels, the allocation-free deposit, the fused x-y transforms) and link
against cuFFT.  Usage: ``python -m paper_1608_00802_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpm.so")
SOURCES = ["pm_api.cu", "pm_kernels_f32.cu", "pm_kernels_f64.cu", "pm_noalloc.cu", "pm_xyfft.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    env = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if env and os.path.isdir(env):
        return env
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("command failed: %s\n%s%s" % (" ".join(cmd), res.stdout, res.stderr))
    return res.stdout + res.stderr


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> str:
    """Compiles libpm.so if a source is newer than it (or `force`).  Extra nvcc
    flags may also come from the PM_EXTRA_NVCC_FLAGS environment variable
    (space separated, e.g. -DPM_ST_PF=6); they always force a rebuild."""
    env_flags = tuple(os.environ.get("PM_EXTRA_NVCC_FLAGS", "").split())
    extra_flags = tuple(extra_flags) + env_flags
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pm.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest and not extra_flags:
        return LIB
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), *extra_flags]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        out = _run([*common, "-c", os.path.join(CSRC, src), "-o", obj])
        return obj, out

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for obj, out in results:
        if verbose and out.strip():
            print(out)
    libdir = os.path.join(home, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(home, "lib")
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-L", libdir, "-lcufft",
          "-Xlinker", "-rpath=" + libdir])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True,
                extra_flags=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
