"""Build the CUDA library libkkt_schur.so in-tree (sm_103a only).

    python -m paper_1907_05420_gb300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkkt_schur.so")
SYM_LIB = os.path.join(OUT_DIR, "libkkt_symbolic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["api.cu", "factor.cu", "tail.cu", "schur.cu", "dense.cu", "solve.cu", "probe.cu", "noalloc.cu", "dense_tc.cu",
      "schur_tc.cu", "shard.cu", "slack.cu", "cumulative.cu"]
CPP = ["symbolic.cpp", "serve.cpp"]
HEADERS = ["handle.h", "symbolic.h", "dense_kernels.cuh", "pivot.cuh", "emu_arith.cuh"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(CSRC, h) for h in HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "kkt_schur.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build_symbolic(force: bool = False) -> str:
    """Host-only inspection library of the symbolic analysis (g++, no CUDA)."""
    srcs = [os.path.join(CSRC, f) for f in ("symbolic.cpp", "symbolic_capi.cpp")]
    deps = srcs + [os.path.join(CSRC, "symbolic.h"),
                   os.path.join(os.path.dirname(HERE), "include", "kkt_symbolic.h")]
    if not force and os.path.exists(SYM_LIB) and all(os.path.getmtime(p) <= os.path.getmtime(SYM_LIB)
                                                    for p in deps):
        return SYM_LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = SYM_LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp] + srcs, check=True)
    os.replace(tmp, SYM_LIB)
    return SYM_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"]
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + common + ["-c", src, "-o", obj]
        else:
            cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", cuda_inc, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    print(build_symbolic(force="--force" in sys.argv))
