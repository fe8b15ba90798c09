"""Compile the CUDA sources into the in-tree shared library ``libpsps.so``.

nvcc cross-compiles for sm_103a (GB300); translation units are compiled in
parallel and linked with ``nvcc -shared``.  No PyTorch headers are involved:
the library is a plain C ABI (``include/mbir.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libpsps.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpsps.so")
    return cand


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


# model_inst.cu instantiates the model kernels of one material count and one
# family per compilation (96 kernel variants in all), so it is compiled once
# per (count, family) pair and the pairs build in parallel.
MODEL_INST = "model_inst.cu"


def units():
    """(source, object name, extra flags) of every compilation."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        if os.path.basename(src) == MODEL_INST:
            for nm in (1, 2, 3, 4):
                for rows in (0, 1):
                    out.append((src, f"{base}_{nm}_{rows}.o", [f"-DPSPS_MODEL_NM={nm}", f"-DPSPS_MODEL_ROWS={rows}"]))
        else:
            out.append((src, base + ".o", []))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(HERE, "..", "include", "mbir.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    objs = []

    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "mbir.h"), __file__]
    t_head = max(os.path.getmtime(h) for h in headers if os.path.exists(h))

    def one(unit):
        src, name, extra = unit
        obj = os.path.join(OUT_DIR, name)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) > max(t_head, os.path.getmtime(src)):
            return obj   # up to date: newer than its source and every header
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        return obj

    # slowest compilations first, so the pool's last worker is not left with one
    todo = sorted(units(), key=lambda u: (os.path.basename(u[0]) != MODEL_INST, u[1]))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(one, todo))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
