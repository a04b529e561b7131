"""Build the ISRS GN CUDA library in-tree for sm_103a (GB300).

Compiles every ``csrc/*.cu`` translation unit in parallel with nvcc and links
``_build/libisrs_gn_<arch>.so``.  No cmake; one ``-gencode``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, f"libisrs_gn_{platform.machine()}.so")
# the bounds-checked debug build (-DISRS_DEBUG): same sources, its own objects
LIB_DEBUG = os.path.join(BUILD, f"libisrs_gn_debug_{platform.machine()}.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the ISRS GN CUDA library cannot be built")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "isrs_gn.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile every csrc/*.cu for sm_103a and link the library; debug=True
    builds the bounds-checked variant (ISRS_DEBUG) beside the release one."""
    os.makedirs(BUILD, exist_ok=True)
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime() and not extra:
        return lib
    cc = nvcc()
    objs = []
    tag = ".debug" if debug else ""
    extra = (*extra, "-DISRS_DEBUG") if debug else tuple(extra)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + f"{tag}.{platform.machine()}.o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for obj, log in ex.map(compile_one, sources()):
            objs.append(obj)
            if verbose and log:
                print(log)
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
