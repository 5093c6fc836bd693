"""Build libdbie.so in-tree for sm_103a (nvcc, one translation unit per process, in parallel)."""
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
LIB = os.path.join(PKG, "libdbie.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "1444",
          f"-I{INCLUDE}", f"-I{CSRC}"]
# Translation units; the lambda-search file is compiled without FMA contraction so the simplex
# arithmetic rounds each operation as written.
UNITS = {
    "capi.cu": [],
    "aux.cu": [],
    "solve.cu": ["-fmad=false"],
    "second_order.cu": ["-fmad=false"],
    "pairsum_f32_val.cu": [],
    "pairsum_f32_obj.cu": [],
    "pairsum_f32_objl.cu": [],
    "pairsum_f32_newton.cu": [],
    "pairsum_f32_hess.cu": [],
    "pairsum_f32_nv.cu": [],
    "pairsum_f32_split.cu": [],
    "pairsum_f64.cu": [],
    "pairsum_ff.cu": [],
    "pairsum_dif.cu": [],
    "vjp.cu": [],
    "noalloc.cu": [],
    "pxe.cu": [],
}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdbie.so")


def _sources_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          extra: list[str] | None = None, lib: str | None = None) -> str:
    """Compile every translation unit and link libdbie.so.  `extra` adds nvcc flags (e.g.
    -D knobs of the pair-sum kernel) and `lib` redirects the output (with its own object dir)."""
    global LIB, BUILD
    if lib is not None:
        LIB, BUILD = lib, lib + ".objs"
    extra = list(extra or [])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(unit):
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *extra, *UNITS[unit], "-c", os.path.join(CSRC, unit), "-o",
               obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    jobs = jobs or min(len(UNITS), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
