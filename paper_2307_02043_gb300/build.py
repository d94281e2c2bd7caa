"""Build libmqnpm.so in-tree for sm_103a.

Every translation unit is compiled in parallel with nvcc (the Green's-apply
passes once per transform length P), then linked into one shared library
under ``paper_2307_02043_gb300/_build``.  A stamp of the sources and flags
skips the build when nothing changed.
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
LIB = os.path.join(BUILD, "libmqnpm.so")

P_VALUES = (16, 24, 32, 48, 64, 96, 128, 192, 256, 320, 384)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-std=c++17", "-O3", ARCH, "-lineinfo", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC", "-I" + CSRC, "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmqnpm")


def _units():
    units = []
    for P in P_VALUES:
        units.append(("green_inst.cu", ["-DMQ_P=%d" % P], "green_P%d.o" % P))
    for name in ("green.cu", "krylov.cu", "wprox_coop.cu", "woodbury.cu", "api.cu", "noalloc.cu", "tune.cu", "detector.cu",
                 "group.cu"):
        units.append((name, [], name.replace(".cu", ".o")))
    units.append(("wprox_coop.cu", ["-DMQ_WP_HIGH"], "wprox_high.o"))   # ranks 9-16 of the prox kernel
    return units


def _stamp() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "mqnpm.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link the library; returns the path of libmqnpm.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_path = os.path.join(BUILD, "stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read().strip() == stamp:
                return LIB
    cc = nvcc()
    jobs = jobs or max(1, min(len(_units()), os.cpu_count() or 4))

    def compile_one(unit):
        src, extra, obj = unit
        cmd = [cc, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-4000:]))
        return os.path.join(BUILD, obj)

    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + ".tmp"
    cmd = [cc, "-shared", ARCH, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
