"""Build the sm_103a shared libraries in-tree (python -m paper_2510_05100_b300.build).

Steps: regenerate the amplitude header from the code generator, compile every
.cu under csrc/ for sm_103a with nvcc and every host .cpp with the C++ compiler,
then link librex_b300.so (the reweighting ABI, include/rex.h) next to this file;
compile csrc/tooling/*.cu into librex_tooling_b300.so (measurement and test
probes, include/rex_tooling.h).  nvcc cross-compiles, so this runs without a GPU.

Objects are rebuilt only when their compile command or one of the files the
compiler read (its dependency file) changed since the last build.
"""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librex_b300.so")
TOOLING_LIB = os.path.join(HERE, "librex_tooling_b300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def tooling_sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "tooling", "*.cu")))


def cxx() -> str:
    return os.environ.get("CXX") or "g++"


def _command(src: str, obj: str, ptxas_info: bool) -> list:
    dep = obj + ".d"
    if src.endswith(".cpp"):   # host-only C++ (the LHE front-end)
        return [cxx(), "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", os.path.join(ROOT, "include"), "-MD", "-MF",
                dep, "-c", "-o", obj, src]
    cmd = [nvcc(), *ARCH, *FLAGS, "-MD", "-MF", dep, "-c", "-o", obj, src]
    if ptxas_info:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def _up_to_date(cmd: list, obj: str) -> bool:
    """True if obj was built by this exact command and no file it depends on is newer."""
    stamp, dep = obj + ".cmd", obj + ".d"
    if not (os.path.exists(obj) and os.path.exists(stamp) and os.path.exists(dep)):
        return False
    if open(stamp).read() != hashlib.sha256(" ".join(cmd).encode()).hexdigest():
        return False
    text = open(dep).read().replace("\\\n", " ")
    files = text.split(":", 1)[1].split() if ":" in text else []
    t_obj = os.path.getmtime(obj)
    return all(os.path.exists(f) and os.path.getmtime(f) <= t_obj for f in files)


def _compile(src: str, obj: str, ptxas_info: bool, force: bool):
    cmd = _command(src, obj, ptxas_info)
    if not force and not ptxas_info and _up_to_date(cmd, obj):
        return cmd, None
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode == 0:
        with open(obj + ".cmd", "w") as f:
            f.write(hashlib.sha256(" ".join(cmd).encode()).hexdigest())
    return cmd, res


def _link(objs: list, lib: str):
    link = [nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lpthread"]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed ({res.returncode}):\n{res.stdout}\n{res.stderr}")


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    """Compile every out-of-date source to an object in parallel, then link librex_b300.so
    and librex_tooling_b300.so."""
    from concurrent.futures import ThreadPoolExecutor

    from .codegen.__main__ import generate

    generate()
    objdir = os.path.join(ROOT, "_build", "obj")
    os.makedirs(os.path.join(objdir, "tooling"), exist_ok=True)
    srcs = sources()
    tsrcs = tooling_sources()
    objs = [os.path.join(objdir, os.path.splitext(os.path.basename(s))[0] + ".o") for s in srcs]
    tobjs = [os.path.join(objdir, "tooling", os.path.splitext(os.path.basename(s))[0] + ".o") for s in tsrcs]
    jobs = list(zip(srcs + tsrcs, objs + tobjs))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda so: _compile(so[0], so[1], ptxas_info, force), jobs))
    for cmd, res in results:
        if res is None:
            continue
        if verbose:
            print(" ".join(cmd))
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed ({res.returncode}):\n{res.stdout}\n{res.stderr}")
        if ptxas_info or verbose:
            sys.stdout.write(res.stdout + res.stderr)
    rebuilt = [res is not None for _, res in results]
    if any(rebuilt[:len(objs)]) or not os.path.exists(LIB):
        _link(objs, LIB)
    if any(rebuilt[len(objs):]) or not os.path.exists(TOOLING_LIB):
        _link(tobjs, TOOLING_LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv, force="--force" in sys.argv)
