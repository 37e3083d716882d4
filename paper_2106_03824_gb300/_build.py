"""Build the CUDA library in-tree: paper_2106_03824_gb300/_lib/libplds_gb300.so.

One nvcc invocation per translation unit (run in parallel), sm_103a only,
then a shared link with the static CUDA runtime.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INC = PKG.parent / "include"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libplds_gb300.so"
SOURCES = ["plds_api.cu", "plds_tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def _flags(src: str):
    # host code: no fused multiply-add contraction (threshold tables in double must round
    # the same way on every host)
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", str(CSRC), "-I", str(INC)]
    if src.endswith(".cu"):
        f += ARCH + ["-lineinfo", "-Xptxas", "-dlcm=cg", "--expt-relaxed-constexpr"]
        if os.environ.get("PLDS_PTXAS_VERBOSE"):
            f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False) -> Path:
    OUT_DIR.mkdir(parents=True, exist_ok=True)
    srcs = [CSRC / s for s in SOURCES]
    deps = srcs + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + [INC / "plds.h"]
    if not force and LIB.exists() and LIB.stat().st_mtime >= max(p.stat().st_mtime for p in deps):
        return LIB
    nvcc = _nvcc()
    objs = [OUT_DIR / (s + ".o") for s in SOURCES]

    def compile_one(i):
        cmd = [nvcc, "-c", str(srcs[i]), "-o", str(objs[i])] + _flags(SOURCES[i])
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {SOURCES[i]}:\n{r.stdout}\n{r.stderr}")
        if r.stderr and (verbose or os.environ.get("PLDS_PTXAS_VERBOSE")):
            print(r.stderr, file=sys.stderr)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(compile_one, range(len(SOURCES))))
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [nvcc, "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + \
          ["-cudart", "static", "-Xcompiler", "-fPIC", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
