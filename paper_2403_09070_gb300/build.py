"""Build libplace3d.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SO = os.path.join(HERE, "libplace3d.so")
UNITS = ["place3d.cu", "tc_gemm.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the place3d CUDA library cannot be built")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libplace3d.so."""
    newest = max(os.path.getmtime(f) for f in _sources())
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    nvcc = _nvcc()
    bdir = os.path.join(os.path.dirname(HERE), "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, u.replace(".cu", ".o")) for u in UNITS]

    def comp(u, o):
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, u), "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        list(ex.map(comp, UNITS, objs))
    tmp = SO + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=False))
