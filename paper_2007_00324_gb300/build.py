"""In-tree build of libgdp.so (nvcc, sm_103a only)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgdp.so")
SOURCES = ["gdp.cu", "gdp_noalloc.cu", "gdp_peak.cu"]
HEADERS = ["gdp_core.cuh", "gdp_pred.cuh", "gdp_kernels.cuh", "gdp_cdt.cuh", "gdp_server.cuh", "gdp_tune.cuh",
           "gdp_flipflop.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "gdp.h")]
    if not force and os.path.exists(LIB):
        mt = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= mt for d in deps):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *srcs]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    extra = os.environ.get("GDP_NVCC_FLAGS", "").split()
    if extra:
        cmd[1:1] = extra
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
