"""Build libpfgpu.so in-tree with nvcc for sm_103a (GB300).

Every ``csrc/*.cu`` file is compiled in parallel to an object, then linked into
``_build/libpfgpu.so``.  A stamp of the sources and flags skips rebuilds that would
produce the same library.  No CMake and no torch extension machinery: the library
has a plain C ABI (``include/pfgpu.h``) and is loaded with ctypes.
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libpfgpu.so")
# The checked variant (-DPF_CHECK): every kernel fills its shared memory with NaN before
# staging, so a read of a slot that staging or an earlier sub-step did not write poisons the
# result and the parity tests see it (compute-sanitizer is not available).
CHECKED_BUILD = os.path.join(BUILD, "checked")
CHECKED_LIB = os.path.join(CHECKED_BUILD, "libpfgpu_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-I", INCLUDE,
              "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpfgpu")


def _cuda_libdir(nvcc: str) -> str:
    """The toolkit directory holding libcufft.so.12 (cuFFT is loaded from there at run time
    if the loader's search path does not have it)."""
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    cands = [os.path.join(root, "lib64"), os.path.join(root, "lib")]
    tdir = os.path.join(root, "targets")
    if os.path.isdir(tdir):
        cands += [os.path.join(tdir, t, "lib") for t in sorted(os.listdir(tdir))]
    for c in cands:
        if os.path.exists(os.path.join(c, "libcufft.so.12")):
            return c
    return ""


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stamp(extra_flags) -> str:
    h = hashlib.sha256()
    for p in sorted(os.listdir(CSRC)) + [os.path.join("..", "..", "include", "pfgpu.h")]:
        full = os.path.normpath(os.path.join(CSRC, p))
        if os.path.isfile(full):
            h.update(p.encode())
            with open(full, "rb") as f:
                h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra_flags)).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile and link the library (checked: the PF_CHECK variant); returns its path."""
    bdir, lib = (CHECKED_BUILD, CHECKED_LIB) if checked else (BUILD, LIB)
    if checked:
        extra_flags = list(extra_flags) + ["-DPF_CHECK"]
    os.makedirs(bdir, exist_ok=True)
    stamp_file = os.path.join(bdir, "stamp.txt")
    stamp = _stamp(list(extra_flags) + [_cuda_libdir(_nvcc())])
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        if open(stamp_file).read().strip() == stamp:
            return lib
    nvcc = _nvcc()
    srcs = _sources()
    extra_flags = list(extra_flags) + [f'-DPF_CUDA_LIBDIR="{_cuda_libdir(nvcc)}"']

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcuda", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        raise RuntimeError(f"link of {os.path.basename(lib)} failed")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp + "\n")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
