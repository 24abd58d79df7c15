"""Build the sm_103a shared library ``_lib/libmfc.so`` in-tree with nvcc.

Each CUDA translation unit compiles in its own nvcc process (in parallel), then one link step
makes the shared library.  Only ``-gencode arch=compute_103a,code=sm_103a`` is emitted.  With
``check_bounds`` the same sources build, with ``-DMFC_CHECK_BOUNDS``, into the debugging library
``_lib/libmfc_check.so`` (element offsets checked in the step kernels, guard regions around every
device buffer).

    python -m paper_1802_07525_gb300.build [--force] [--ptxas-verbose] [--check-bounds]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libmfc.so")
LIB_CHECK = os.path.join(OUT_DIR, "libmfc_check.so")
OBJ_DIR = os.path.join(HERE, "_build")
OBJ_DIR_CHECK = os.path.join(HERE, "_build_check")
SOURCES = ["lbm2d_f32.cu", "lbm2d_f16.cu", "lbm3d_f32.cu", "lbm3d_f16.cu", "lbm2d9_f32.cu",
           "lbm2d9_f16.cu", "lbm2d_f64.cu", "lbm3d_f64.cu", "lbm2d9_f64.cu", "runtime.cu", "batch.cu",
           "noalloc.cu", "electro.cu", "agent.cu", "slab.cu"]
HEADERS = ["lbm_lattice.cuh", "lbm_kernels.cuh", "lbm_pair.cuh", "lbm_aux.cuh", "lbm_launch.cuh", "mfc_internal.h",
           "runtime.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmfc")


def _flags(verbose: bool, relative: bool = False, check_bounds: bool = False):
    """nvcc flags; with ``relative`` the include directories are named relative to the repository
    root, so that a digest of the flags is the same in every checkout."""
    inc = "include" if relative else os.path.join(ROOT, "include")
    src = os.path.relpath(CSRC, ROOT) if relative else CSRC
    f = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", inc, "-I", src] + ARCH
    if check_bounds:
        f += ["-DMFC_CHECK_BOUNDS"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _digest(verbose: bool, check_bounds: bool = False) -> str:
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "mfc.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(_flags(verbose, check_bounds=check_bounds)).encode())
    return h.hexdigest()


# The files each step-kernel translation unit compiles from (the TU and the headers it includes).
KERNEL_TU_FILES = ["lbm_launch.cuh", "mfc_internal.h", "lbm_kernels.cuh", "lbm_lattice.cuh", "lbm_pair.cuh"]


def kernel_digest(tu: str) -> str:
    """Digest of one step-kernel translation unit: the contents of its source and of the headers
    it includes, and the flags with repository-relative paths (no path of the machine enters it).
    A profile taken on a build with the same digest was taken on the same kernel code."""
    h = hashlib.sha256()
    for name in [tu] + KERNEL_TU_FILES:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(_flags(False, relative=True)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, quiet: bool = True,
          check_bounds: bool = False) -> str:
    """Compile (if sources changed) and return the path of libmfc.so (libmfc_check.so with
    check_bounds)."""
    lib_path = LIB_CHECK if check_bounds else LIB
    obj_dir = OBJ_DIR_CHECK if check_bounds else OBJ_DIR
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    stamp = lib_path.replace(".so", ".sha256")
    dig = _digest(verbose, check_bounds)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return lib_path
    cc = nvcc()
    flags = _flags(verbose, check_bounds=check_bounds)

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if not quiet or verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["--cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return lib_path


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-verbose", action="store_true")
    ap.add_argument("--check-bounds", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.ptxas_verbose, quiet=False, check_bounds=a.check_bounds))
