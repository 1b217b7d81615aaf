"""Build libsph.so (the CUDA library behind include/sph.h) for sm_103a.

Each translation unit under csrc/ is compiled in parallel with nvcc and the
objects are linked into ``paper_1603_02421_gb300/libsph.so``, in the source
tree.  The CUDA runtime is linked statically, so the library needs only the
driver at run time.  Host code is compiled with -ffp-contract=off, so the
few host-side FP64 formulas that must agree bit for bit with a plain
evaluation (inflow layer positions, thresholds) are not fused.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsph.so")
# the bounds-check build (SPH_BOUNDS_CHECK): the same library with every
# particle index met by the neighbour walks and the network's gathers checked
# against the capacity (ERR_BOUNDS, SPH_ERR_STATE); a diagnostic, not the
# product path
BUILD_BOUNDS = os.path.join(PKG, "_build_bounds")
LIB_BOUNDS = os.path.join(PKG, "libsph_bounds.so")
SOURCES = ["sph_api.cu", "sph_neighbour.cu", "sph_sweeps.cu", "sph_noalloc.cu", "sph_mpnn.cu",
           "sph_mpnn_tc.cu", "sph_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                   "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "sph.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), bounds_check: bool = False) -> str:
    """Compile and link libsph.so (bounds_check: libsph_bounds.so, with
    SPH_BOUNDS_CHECK defined); returns its path."""
    lib = LIB_BOUNDS if bounds_check else LIB
    bdir = BUILD_BOUNDS if bounds_check else BUILD
    if not force and not extra and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = _flags() + list(extra) + (["-DSPH_BOUNDS_CHECK"] if bounds_check else [])

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for obj, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    extra = sys.argv[1:]
    print(build(force=True, verbose=True, extra=extra))
