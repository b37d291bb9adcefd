"""Build libckpp.so (the CUDA library behind include/ckpp.h, and the served
form's host runtime behind include/ckpp_serve.h) for sm_103a.

Each ``csrc/*.cu`` / ``csrc/*.cpp`` file is compiled by nvcc in parallel into ``_build/`` and
linked into ``libckpp.so`` next to this file. A rebuild happens only when a
source or header is newer than the library (or ``force``).
"""

from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libckpp.so")
WL_LIB = os.path.join(HERE, "libckpp_workload.so")
HEADER = os.path.join(ROOT, "include", "ckpp.h")
SERVE_HEADER = os.path.join(ROOT, "include", "ckpp_serve.h")
WL_HEADER = os.path.join(ROOT, "include", "ckpp_workload.h")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_lib(lib: str, sources: list[str], headers: list[str], objdir: str, force: bool, verbose: bool) -> str:
    if not force and not _stale(lib, sources + headers + [__file__]):
        return lib
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(sources))) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libckpp.so (the method) and libckpp_workload.so (device-side
    synthetic traffic); returns the path of libckpp.so."""
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))) + [HEADER,
                                                                                                        SERVE_HEADER]
    wl_sources = sorted(glob.glob(os.path.join(CSRC, "workload", "*.cu")))
    with ThreadPoolExecutor(max_workers=2) as ex:
        f1 = ex.submit(_build_lib, LIB, sources, headers, BUILD, force, verbose)
        f2 = ex.submit(_build_lib, WL_LIB, wl_sources, [WL_HEADER], os.path.join(BUILD, "workload"), force, verbose)
        f2.result()
        return f1.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
