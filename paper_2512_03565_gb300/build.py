"""Builds the CUDA library libljgb.so in-tree (paper_2512_03565_gb300/_build/).

Every translation unit under csrc/ is compiled for sm_103a (GB300) in
parallel with nvcc and linked into one shared library that exports the C ABI
declared in include/ljgb.h.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
# LJGB_CHECKS=1: a separate build whose kernels check every index they read
# from data (list entries, segments, cluster entries, permutation slots) and
# set a status bit instead of making the access (LJ_ERR_CUDA "device index
# check failed" at the next status read).
CHECKS = os.environ.get("LJGB_CHECKS", "0") not in ("", "0")
OUT = os.path.join(HERE, "_build_checks" if CHECKS else "_build")
LIB = os.path.join(OUT, "libljgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"] + (["-DLJGB_CHECKS=1"] if CHECKS else [])


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "ljgb.h")]
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, hdr_mtime: float, verbose: bool, out: str, flags: list[str]) -> str:
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime):
        return obj
    cmd = [NVCC, *ARCH, *flags, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None, out: str | None = None,
          host_flags: tuple[str, ...] = ()) -> str:
    """Compiles into `out` (default: the in-tree build folder) and returns the
    library's path.  `host_flags` go to the host compiler of every unit and of
    the link (e.g. sanitizers for the host-side code); a build with them must
    name its own `out`."""
    if host_flags and out is None:
        raise ValueError("a build with host_flags needs its own output folder")
    out = out or OUT
    lib = os.path.join(out, "libljgb.so")
    os.makedirs(out, exist_ok=True)
    xhost = [a for f in host_flags for a in ("-Xcompiler", f)]
    flags = FLAGS + xhost
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hm = _headers_mtime()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, hm, verbose, out, flags), srcs))
    if (not os.path.exists(lib)) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        cmd = [NVCC, *ARCH, *xhost, "-shared", "-o", lib + ".tmp", *objs, "-ldl"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
