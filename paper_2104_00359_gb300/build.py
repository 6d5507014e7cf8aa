"""Build the CUDA shading library ``libshshadow.so`` in-tree (sm_103a).

Compiles ``csrc/shs_api.cu`` and one object of ``csrc/shs_kern.cu`` per band
count (-DSHS_NB=1..8) in parallel with nvcc, then links them into
``paper_2104_00359_gb300/lib/libshshadow.so``.  Objects are cached under
``_build/`` and rebuilt when a source or header is newer.
"""

from __future__ import annotations

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
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libshshadow.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
BANDS = (1, 2, 3, 4, 5, 6, 7, 8)


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libshshadow")
    return exe


def _deps():
    out = [os.path.join(INCLUDE, "shs.h")]
    for d, _, files in os.walk(CSRC):
        out += [os.path.join(d, f) for f in files if f.endswith((".cu", ".cuh", ".h"))]
    return out


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _tune_defines():
    """Optional -D tuning flags from SHS_TUNE="NAME=V,NAME=V" (e.g. register
    caps for launch-bound experiments)."""
    spec = os.environ.get("SHS_TUNE", "").strip()
    return [f"-D{kv.strip()}" for kv in spec.split(",") if kv.strip()]


def _flags():
    # -ftz=true: float32 denormals flush to zero, so rsqrt/rcp map to single
    # MUFU instructions (no denormal fix-up code); the path never produces
    # values below 1e-38 that matter to the result.
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-ftz=true",
                   "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _compile(src, obj, defines, log):
    cmd = [nvcc()] + _flags() + ["-Xptxas", "-v"] + defines + _tune_defines() + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as fh:
        fh.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr[-4000:]}")
    return obj


def build(verbose=False, jobs=None):
    """Compile (if stale) and link the library; returns its path."""
    sys.path.insert(0, CSRC)
    try:
        import gen_tables
        if gen_tables.main(["--check"]) != 0:
            gen_tables.main([])
    finally:
        sys.path.remove(CSRC)
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    deps = _deps()
    units = [(os.path.join(CSRC, "shs_api.cu"), os.path.join(BUILD, "shs_api.o"), []),
             (os.path.join(CSRC, "shs_noalloc.cu"), os.path.join(BUILD, "shs_noalloc.o"), []),
             (os.path.join(CSRC, "shs_tc.cu"), os.path.join(BUILD, "shs_tc.o"), []),
             (os.path.join(CSRC, "shs_env.cu"), os.path.join(BUILD, "shs_env.o"), []),
             (os.path.join(CSRC, "shs_raster.cu"), os.path.join(BUILD, "shs_raster.o"), []),
             (os.path.join(CSRC, "shs_diag.cu"), os.path.join(BUILD, "shs_diag.o"), []),
             (os.path.join(CSRC, "shs_chain.cu"), os.path.join(BUILD, "shs_chain.o"), []),
             (os.path.join(CSRC, "shs_tail_tc.cu"), os.path.join(BUILD, "shs_tail_tc.o"), ["-DSHS_NB=8"])]
    for n in BANDS:
        units.append((os.path.join(CSRC, "shs_kern.cu"), os.path.join(BUILD, f"shs_kern_{n}.o"),
                      [f"-DSHS_NB={n}"]))
    todo = [u for u in units if _stale(u[1], deps)]
    if todo:
        jobs = jobs or min(len(todo), max(1, os.cpu_count() or 1))
        with ThreadPoolExecutor(jobs) as ex:
            futs = [ex.submit(_compile, s, o, d, o[:-2] + ".log") for s, o, d in todo]
            for f in futs:
                obj = f.result()
                if verbose:
                    print("built", os.path.basename(obj))
    objs = [u[1] for u in units]
    if _stale(LIB, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr[-4000:])
        if verbose:
            print("linked", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
