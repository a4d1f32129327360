"""Build libcpct.so (the CUDA library behind include/cpct.h) for sm_103a.

Compiles every ``csrc/*.cu`` translation unit in parallel with nvcc and links
them into ``_lib/libcpct.so`` inside the package (in-tree, git-ignored).  A
hash of the sources and flags is stored next to the library so that an
unchanged tree is not rebuilt.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libcpct.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
    "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
    "-I", INCLUDE, "-I", CSRC,
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcpct")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _hash_files(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())  # names, not paths: equal on every machine
        with open(f, "rb") as fh:
            h.update(fh.read())
    # flags with the include directories by name: the repository's location
    # differs between machines
    h.update(" ".join(os.path.basename(f) if os.path.isabs(f) else f for f in NVCC_FLAGS).encode())
    return h.hexdigest()


def _digest() -> str:
    return _hash_files(sources() + sorted(
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))
    ) + [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE))])


def source_digest() -> str:
    """SHA-256 of the CUDA sources, headers and build flags (identifies a kernel version)."""
    return _digest()


# files that define the Radon operator kernels (kernels, their headers, and
# the plan and bin-plan builders whose tables and bins they read)
RADON_FILES = ("radon.cu", "plan.cu", "bins.cu", "bins.cuh", "common.cuh", "fft.cuh")


def radon_digest() -> str:
    """SHA-256 of the Radon operator's sources and build flags: identifies the
    kernel version an ncu summary of an operator kernel was taken on."""
    return _hash_files([os.path.join(CSRC, f) for f in RADON_FILES])


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libcpct.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "libcpct.sha256")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, "-c", src, "-o", obj] + NVCC_FLAGS
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
