"""Build libbshuffle.so for sm_103a with nvcc, in-tree.

Each translation unit in ``csrc/`` is compiled in parallel, then linked into
``paper_2106_06161_gb300/_build/libbshuffle.so`` with the CUDA runtime linked
statically.  A hash of the sources and flags skips rebuilds that would change
nothing.  Usage: ``python -m paper_2106_06161_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libbshuffle.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbshuffle")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _fingerprint(sources: list[str]) -> str:
    h = hashlib.sha256()
    files = sources + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")))
    files.append(os.path.join(ROOT, "include", "bshuffle.h"))
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + [f for f in NVCC_FLAGS if not os.path.isabs(f)]).encode())
    return h.hexdigest()


def kernel_fingerprint(source: str) -> str:
    """Hash of one kernel translation unit, every csrc header and the flags."""
    h = hashlib.sha256()
    headers = sorted(os.path.basename(f) for f in glob.glob(os.path.join(CSRC, "*.cuh")) +
                     glob.glob(os.path.join(CSRC, "*.h")))
    for name in [source] + headers:
        h.update(name.encode())
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + [f for f in NVCC_FLAGS if not os.path.isabs(f)]).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, defines: tuple = (), build_dir: str | None = None) -> str:
    """Compile and link the library; returns the path of the shared object.

    `defines` (e.g. ("BSHUFFLE_LOOKBACK_CLOCKS=1",)) builds a variant of the
    library; give it its own `build_dir` so that the default build stays."""
    bdir = BUILD_DIR if build_dir is None else build_dir
    lib_path = os.path.join(bdir, LIB_NAME)
    extra = [f"-D{d}" for d in defines]
    os.makedirs(bdir, exist_ok=True)
    sources = _sources()
    stamp_path = os.path.join(bdir, "stamp.txt")
    fp = _fingerprint(sources) + ("|" + ",".join(defines) if defines else "")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            if fh.read().strip() == fp:
                return lib_path
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(sources))) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = lib_path + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"linking {LIB_NAME} failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp_path, "w") as fh:
        fh.write(fp)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
