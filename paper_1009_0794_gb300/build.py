"""Build libldni.so in-tree: every ``csrc/*.cu`` compiled for sm_103a in
parallel, then linked into ``_build/libldni.so``.

    python -m paper_1009_0794_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
# LDNI_BUILD_DIR puts a variant build (other LDNI_EXTRA_NVCC_FLAGS, e.g. the
# checked build) beside the default one instead of over it.
BUILD = os.environ.get("LDNI_BUILD_DIR") or os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libldni.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the LDNI CUDA library cannot be built")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(INCLUDE, "ldni.h"))
    return sorted(hs)


def _stamp(units=None) -> str:
    """Hash of the sources (every .cu file, or only `units`, file names in
    csrc), every header and the flags: it names the build, and, per unit,
    the code of the kernels a recorded profile was taken from."""
    h = hashlib.sha256()
    srcs = _sources() if units is None else sorted(os.path.join(CSRC, u) for u in units)
    for f in srcs + _headers():
        with open(f, "rb") as fh:
            h.update(os.path.relpath(f, ROOT).encode())  # the same on every checkout
            h.update(fh.read())
    # include directories relative to the repository, like the file names
    flags = [os.path.relpath(f, ROOT) if os.path.isabs(f) else f for f in NVCC_FLAGS]
    h.update(" ".join(ARCH + flags).encode())
    return h.hexdigest()


def _compile(nvcc: str, src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link libldni.so unless an up-to-date build exists.  extra:
    more nvcc flags (also taken, space-separated, from LDNI_EXTRA_NVCC_FLAGS)."""
    extra = tuple(extra) + tuple(os.environ.get("LDNI_EXTRA_NVCC_FLAGS", "").split())
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "stamp.txt")
    stamp = _stamp() + "|" + " ".join(extra)
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read() == stamp:
                return LIB
    nvcc = _nvcc()
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, list(extra)), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
