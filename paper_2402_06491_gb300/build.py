"""Build libgrt.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel, then linked with the static CUDA
runtime.  The library lands next to this file; nothing is installed.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libgrt.so")

# (source, object name, extra nvcc flags): grt_walk_u0.cu is compiled once per launch shape
SOURCES = [("grt_api.cu", "grt_api", []), ("grt_walk.cu", "grt_walk", []), ("grt_walk_feat.cu", "grt_walk_feat", []),
           ("grt_trees.cu", "grt_trees", []), ("grt_finalize.cu", "grt_finalize", []),
           ("grt_server.cu", "grt_server", []), ("grt_pdd.cu", "grt_pdd", []), ("grt_plain.cu", "grt_plain", [])]
for _w, _s in ((4, 0), (4, 3), (8, 0), (8, 3)):
    SOURCES.append(("grt_walk_u0.cu", f"grt_walk_u0_w{_w}s{_s}",
                    [f"-DGRT_U0_FN=launch_walk_u0_w{_w}s{_s}", f"-DGRT_U0_WARPS={_w}", f"-DGRT_U0_SLEV={_s}"]))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list:
    out = [os.path.join(INCLUDE, "grt.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def _stale(target: str, deps: list) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA translation unit and link libgrt.so; returns its path."""
    deps = _deps()
    if not force and not ptxas_info and not _stale(LIB_PATH, deps):
        return LIB_PATH
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(entry):
        src, name, defs = entry
        obj = os.path.join(BUILD_DIR, name + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
