"""Build libstm.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel: the residual kernels once per
spatial degree (residual_inst.cu with -DSTM_P=0..7), the Krylov kernels and
the C ABI.  Objects go to _build/ next to this file; the library to
paper_1307_5310_gb300/libstm.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    units = []
    for p in range(8):
        units.append(("residual_inst.cu", f"residual_p{p}.o", [f"-DSTM_P={p}"]))
    for src in ("krylov.cu", "stm_capi.cu", "stm_noalloc.cu", "load.cu", "curved.cu", "curved_tc.cu", "hp.cu",
                "server.cu"):
        units.append((src, src.replace(".cu", ".o"), []))
    return units


def _sources_mtime() -> float:
    m = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return max(m, os.path.getmtime(__file__))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if needed) and return the path of libstm.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cmds = []
    for src, obj, extra in _units():
        cmds.append([nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)])
    jobs = jobs or min(len(cmds), os.cpu_count() or 4)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(jobs) as ex:
        list(ex.map(run, cmds))
    objs = [os.path.join(BUILD, obj) for _, obj, _ in _units()]
    tmp = LIB + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
