"""Build libpichol.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel to an object file under
``_build/``; the objects are linked into ``paper_1404_0466_gb300/libpichol.so``
with the CUDA runtime linked statically, so the library loads (and exports its
symbols) on a machine without a GPU driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import pathlib
import shutil
import subprocess
import sys

PKG = pathlib.Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libpichol.so"
# the bounds-checked variant (-DPICHOL_DEBUG: guard bands after every
# workspace section, checked by pichol_get_info)
BUILD_DEBUG = PKG / "_build_debug"
LIB_DEBUG = PKG / "libpichol_debug.so"
SOURCES = ["api.cu", "gram.cu", "chol.cu", "fit.cu", "solve.cu", "tc_gemm.cu", "grad.cu", "batch.cu", "mchol.cu", "pinrmse.cu", "resid.cu", "solve_single.cu", "probe.cu", "resid_tc.cu", "chol_tc.cu", "solve_tc.cu", "solve_wave.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: pathlib.Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> pathlib.Path:
    """Compile the library (``debug``: the bounds-checked variant) and return its path."""
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    extra = ["-DPICHOL_DEBUG"] if debug else []
    bdir.mkdir(exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + [PKG.parent / "include" / "pichol.h"]
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = CSRC / src
        o = bdir / (src + ".o")
        if force or _stale(o, [s] + headers):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        tmp = o.with_suffix(f".{os.getpid()}.tmp.o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", str(s), "-o", str(tmp)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s.name}:\n{r.stderr}")
        os.replace(tmp, o)
        return s.name, r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for name, err in ex.map(compile_one, jobs):
                if verbose:
                    print(f"compiled {name}", err, file=sys.stderr)
    objs = [bdir / (s + ".o") for s in SOURCES]
    if force or jobs or _stale(lib, objs):
        tmp = PKG / f"{lib.stem}.{os.getpid()}.tmp.so"
        cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
