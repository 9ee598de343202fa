"""Build libprngd.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel, then linked into
``paper_1401_8230_gb300/lib/libprngd.so``. CUDA's runtime is linked statically; the
tensor-map encoder is looked up through the runtime, so libcuda is not a link dependency.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(HERE, "lib")
LIB_PATH = os.path.join(LIB_DIR, "libprngd.so")
OBJ_DIR = os.path.join(HERE, "_build")

SOURCES = ["prngd.cu", "prngd_io.cu", "prngd_stats.cu", "prngd_noalloc.cu", "prngd_batch.cu", "prngd_serve.cpp",
           "prngd_modes.cu", "prngd_modes_fast.cu", "prngd_jump.cu",
           "prngd_mrg.cu", "prngd_convert.cu"]
# (object, source, extra flags): one source compiled once per w
VARIANTS = [(f"prngd_batch_modes_w{w}", "prngd_batch_modes.cu", [f"-DPRNGD_ANY_MODE_W={w}"]) for w in (32, 24, 0)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libprngd")
    return cand


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= _newest_input():
        return LIB_PATH
    os.makedirs(OBJ_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    cc = nvcc()

    units = [(os.path.splitext(src)[0], src, []) for src in SOURCES] + VARIANTS

    def compile_one(unit) -> str:
        name, src, extra = unit
        obj = os.path.join(OBJ_DIR, name + ".o")  # .cpp: host-only, same flags
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
