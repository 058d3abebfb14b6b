"""Builds libtpcf.so (the CUDA estimator behind include/tpcf.h) in the package
directory: one nvcc process per translation unit, run in parallel, for sm_103a
only, then one shared-library link."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtpcf.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-v", "-I", os.path.join(HERE, "..", "include")]


# compiled once per l_max with -DTPCF_LMAX=n (the pair-stage kernels)
PER_LMAX = "k_pairs_inst.cu"
MAX_LMAX = 6


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object, extra flags) for every translation unit."""
    out = []
    for src in _sources():
        base = os.path.basename(src)
        if base == PER_LMAX:
            for l in range(MAX_LMAX + 1):
                out.append((src, os.path.join(OBJ, "%s.l%d.o" % (base, l)), ["-DTPCF_LMAX=%d" % l]))
        else:
            out.append((src, os.path.join(OBJ, base + ".o"), []))
    return out


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(HERE, "..", "include", "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(unit) -> tuple[str, str]:
    src, obj, extra = unit
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every .cu under csrc/ for sm_103a and link libtpcf.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    t0 = time.time()
    units = _units()
    jobs = jobs or min(len(units), max(2, os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(_compile, units))
    with open(os.path.join(OBJ, "ptxas.log"), "w") as f:
        for obj, log in results:
            f.write("== %s\n%s\n" % (obj, log))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("built %s in %.1fs" % (LIB, time.time() - t0), file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
