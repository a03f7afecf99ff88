"""Build libletkf.so (CUDA, sm_103a) in-tree with nvcc.

``python -m paper_1408_7069_gb300.build`` or ``build_library()``. The
translation units compile in parallel; the shared object lands next to this
file, where ``paper_1408_7069_gb300.letkf`` loads it from.
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
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libletkf.so")
PHASE_LIB = os.path.join(PKG, "libletkf_phase.so")
SOURCES = ["letkf_api.cu", "letkf_kernels.cu", "letkf_analysis.cu", "letkf_adjoint.cu", "letkf_pair.cu",
           "letkf_node64.cu", "letkf_peaks.cu", "letkf_domains.cu",
           "letkf_dm.cu", "letkf_global.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libletkf.so")
    return cand


def build_library(verbose: bool = False, ptxas_info: bool = False,
                  phase_clocks: bool = False) -> str:
    """Compile the library; ``phase_clocks`` builds the instrumented variant
    (per-phase cycle counts of the FP32 analysis kernel) as libletkf_phase.so."""
    bdir = os.path.join(BUILD, "phase") if phase_clocks else BUILD
    out = PHASE_LIB if phase_clocks else LIB
    os.makedirs(bdir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
             "--expt-relaxed-constexpr"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    if phase_clocks:
        flags += ["-DLK_PHASE_CLOCKS"]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for obj, log in results:
            if log.strip():
                print(log, file=sys.stderr)
    tmp = out + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_library(verbose=True, ptxas_info="-v" in sys.argv,
                        phase_clocks="--phase-clocks" in sys.argv))
