"""Builds librbffd.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each .cu translation unit is compiled in parallel, then linked into one
shared library with the CUDA runtime linked statically.  A stamp of the
sources and flags skips the build when nothing changed.

build(checked=True) makes the bounds-checked variant, librbffd_checked.so
(-DRBFFD_CHECKED: every computed index is tested before its access and a
violation is recorded instead of performed); the package loads it instead of
librbffd.so when the environment sets RBFFD_CHECKED=1.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(REPO_DIR, "include")
LIB_DIR = os.path.join(PKG_DIR, "lib")
LIB_PATH = os.path.join(LIB_DIR, "librbffd.so")
CHECKED_LIB_PATH = os.path.join(LIB_DIR, "librbffd_checked.so")
OBJ_DIR = os.path.join(PKG_DIR, "_build")
CHECKED_FLAGS = ["-DRBFFD_CHECKED"]

SOURCES = ["api.cu", "knn.cu", "weights.cu", "assemble.cu", "krylov.cu", "batched.cu", "mg.cu", "mg_batch.cu",
           "explicit.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def _nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librbffd")


def lib_path(checked: bool = False) -> str:
    return CHECKED_LIB_PATH if checked else LIB_PATH


def _stamp(extra) -> str:
    h = hashlib.sha256()
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra)).encode())
    for d, names in ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, sorted(os.listdir(INCLUDE)))):
        for nm in names:
            p = os.path.join(d, nm)
            if os.path.isfile(p):
                h.update(nm.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=None, checked: bool = False) -> str:
    """Compile and link the library (the bounds-checked variant when
    `checked`); returns its path."""
    extra = (CHECKED_FLAGS if checked else []) + list(extra_flags or [])
    lib = lib_path(checked)
    obj_dir = os.path.join(OBJ_DIR, "checked") if checked else OBJ_DIR
    os.makedirs(LIB_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    stamp = _stamp(extra)
    stamp_path = lib + ".stamp"
    if not force and os.path.exists(lib) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read().strip() == stamp:
                return lib
    nvcc = _nvcc()
    flags = ARCH + NVCC_FLAGS + ["-I", INCLUDE, "-I", CSRC] + extra

    def compile_one(src: str) -> str:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
