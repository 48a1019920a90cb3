"""Build the sm_103a shared library librex_b300.so in-tree (python -m paper_2510_05100_b300.build).

Steps: regenerate the amplitude header from the code generator, compile every
.cu under csrc/ for sm_103a with nvcc and every host .cpp with the C++ compiler,
then link one shared library next to this file.  nvcc cross-compiles, so this
runs without a GPU.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librex_b300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def cxx() -> str:
    return os.environ.get("CXX") or "g++"


def _compile(src: str, obj: str, ptxas_info: bool):
    if src.endswith(".cpp"):   # host-only C++ (the LHE front-end)
        cmd = [cxx(), "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", os.path.join(ROOT, "include"), "-c", "-o", obj,
               src]
        return cmd, subprocess.run(cmd, capture_output=True, text=True)
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", "-o", obj, src]
    if ptxas_info:
        cmd.insert(1, "-Xptxas=-v")
    return cmd, subprocess.run(cmd, capture_output=True, text=True)


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every csrc/*.cu to an object in parallel, then link librex_b300.so."""
    from concurrent.futures import ThreadPoolExecutor

    from .codegen.__main__ import generate

    generate()
    objdir = os.path.join(ROOT, "_build", "obj")
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(objdir, os.path.splitext(os.path.basename(s))[0] + ".o") for s in srcs]
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda so: _compile(so[0], so[1], ptxas_info), zip(srcs, objs)))
    for cmd, res in results:
        if verbose:
            print(" ".join(cmd))
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed ({res.returncode}):\n{res.stdout}\n{res.stderr}")
        if ptxas_info or verbose:
            sys.stdout.write(res.stdout + res.stderr)
    link = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lpthread"]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed ({res.returncode}):\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
