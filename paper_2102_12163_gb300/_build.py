"""In-tree build of the CUDA library (sm_103a only) with nvcc.

Every ``csrc/*.cu`` is compiled in parallel into an object file and linked into
``libmrlbm.so`` beside this file.  A rebuild happens only when a source or
header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libmrlbm.so")
PROF_LIB = os.path.join(HERE, "libmrlbm_prof.so")  # with per-phase clock timers
BUILD = os.path.join(HERE, "_build")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without fused multiply-add contraction (GCC contracts by default on
# aarch64, not on x86-64), so host-computed constants (M^-1 of the D1Q3 / D1Q5
# schemes, the scheme constants) are the same on both machines
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", f"-I{INCLUDE}"]


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(profile: bool = False) -> bool:
    lib = PROF_LIB if profile else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, profile: bool = False) -> str:
    """Build libmrlbm.so, or with profile=True the phase-timer variant."""
    lib = PROF_LIB if profile else LIB
    if not force and up_to_date(profile):
        return lib
    bdir = BUILD + ("_prof" if profile else "")
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    extra = ["-DMRG_PHASE_TIMERS"] if profile else []

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    workers = max(1, min(len(srcs), os.cpu_count() or 4))
    with ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib
