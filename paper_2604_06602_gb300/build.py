"""Builds libumi.so in-tree: every .cu under csrc/ compiled for sm_103a only.

Translation units compile in parallel (a few seconds each) and are linked
with the static CUDA runtime into ``paper_2604_06602_gb300/libumi.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build", platform.machine())
LIB = os.path.join(PKG, "libumi.so")
STAMP = LIB + ".arch"
# The checked build (UMI_CHECKED: index checks in every kernel, see umi.h).
CHECKED_LIB = os.path.join(PKG, "libumi_checked.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libumi")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    files = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    files.append(os.path.join(ROOT, "include", "umi.h"))
    files.append(os.path.abspath(__file__))
    return files


def _paths(checked: bool):
    lib = CHECKED_LIB if checked else LIB
    return lib, lib + ".arch", BUILD + ("-checked" if checked else "")


def up_to_date(checked: bool = False) -> bool:
    lib, stamp, _ = _paths(checked)
    if not (os.path.exists(lib) and os.path.exists(stamp)):
        return False
    if open(stamp).read().strip() != platform.machine():
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          checked: bool = False) -> str:
    """Compile and link libumi.so (libumi_checked.so with `checked`); returns its path."""
    lib, stamp, bdir = _paths(checked)
    if not force and up_to_date(checked):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    srcs = sources()
    extra = ["-DUMI_CHECKED"] if checked else []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [cc] + ARCH_FLAGS + CFLAGS + extra + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            print(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc] + ARCH_FLAGS + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(platform.machine() + "\n")
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
