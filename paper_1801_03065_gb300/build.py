"""Builds the CUDA library libkkspgemm.so in-tree for sm_103a (GB300).

Each translation unit compiles in parallel with nvcc; the objects link into
``paper_1801_03065_gb300/_lib/libkkspgemm.so`` with the CUDA runtime linked
statically, so the library loads next to any PyTorch build.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libkkspgemm.so")

SOURCES = ["kks_prep.cu", "kks_symbolic.cu", "kks_numeric.cu", "kks_masked.cu", "kks_api.cu", "kks_noalloc.cu", "kks_rap.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "--extended-lambda", "-lineinfo", "-Xcompiler", "-fPIC",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkkspgemm")
    return found


# The sources that a numeric kernel is compiled from and launched by: a
# profile record of a numeric kernel stays valid while these are unchanged.
NUMERIC_SOURCES = ["kks_api.cu", "kks_device.cuh", "kks_internal.h", "kks_numeric.cu"]


def _digest(names=None) -> str:
    """SHA-256 of the library sources (all of csrc/ and the header, or only the
    csrc/ files in names) and of the compiler flags."""
    h = hashlib.sha256()
    groups = ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, ["kkspgemm.h"])) if names is None else \
        ((CSRC, sorted(names)),)
    for d, names in groups:
        for n in names:
            p = os.path.join(d, n)
            if os.path.isfile(p):
                h.update(n.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    # flags without the include directories, whose absolute paths depend on
    # where the repository sits
    h.update(" ".join(ARCH + [f for f in FLAGS if not f.startswith("-I")]).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "build.sha256")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
