"""Build the CUDA library ``libubs.so`` in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel; preprocess.cu gets the float32
rule set's flags (no FMA contraction, correctly rounded division and square
root, no flush-to-zero).  Objects go to ``_build/``, the library next to this
file.  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libubs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
SPEC_FLAGS = ["--fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]
UNITS = {
    "preprocess.cu": SPEC_FLAGS,
    "sort.cu": [],
    "render.cu": [],
    "prim_backward.cu": [],
    "abi.cu": [],
    "noalloc.cu": [],
    "train.cu": [],
    "mcmc.cu": [],
}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libubs.so")
    return path


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def one(item):
        name, extra = item
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, name), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(one, UNITS.items()))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_sanitized(out_dir: str) -> str:
    """The same library with its host code under AddressSanitizer and
    UndefinedBehaviorSanitizer (device code unchanged), for host-side tests of
    the argument checks and layout arithmetic; built into out_dir.  Loading it
    needs the sanitizer runtimes preloaded (LD_PRELOAD)."""
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    san = ["-Xcompiler", "-fPIC,-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer"]
    common = [a for a in COMMON if a not in ("-Xcompiler", "-fPIC")]

    def one(item):
        name, extra = item
        obj = os.path.join(out_dir, name.replace(".cu", ".o"))
        r = subprocess.run([cc, *ARCH, *common, *san, *extra, "-c", os.path.join(CSRC, name), "-o", obj],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS.items()))
    lib = os.path.join(out_dir, "libubs_sanitized.so")
    r = subprocess.run([cc, *ARCH, "-shared", "-Xcompiler", "-fsanitize=address,-fsanitize=undefined", "-o", lib,
                        *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
