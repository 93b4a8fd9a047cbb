"""Build of the sm_103a shared library ``libalm_gb300.so`` (in-tree, no cmake).

Every translation unit is compiled in parallel with nvcc for sm_103a only, then
linked into one shared library next to this file.  Run ``python -m
paper_2505_15775_gb300.build`` or call :func:`build`.
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
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libalm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["pattern.cpp", "kernels_sparse.cu", "kernels_inner.cu", "kernels_growth.cu", "kernels_lanczos.cu", "alm_api.cu", "noalloc.cu", "kernels_batch.cu",
           "kernels_gnn.cu", "gnn_api.cu",
           "batch_api.cu"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _flags() -> list[str]:
    return ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
            "-I", CSRC, "--expt-relaxed-constexpr"]


# translation units compiled once per precision (float and double objects built in parallel)
SPLIT = {"kernels_sparse.cu", "kernels_inner.cu"}


def _units() -> list[tuple[str, str | None]]:
    out = []
    for s in SOURCES:
        if s in SPLIT:
            out += [(s, "1"), (s, "2")]
        else:
            out.append((s, None))
    return out


def _compile(src: str, verbose_ptxas: bool, only: str | None = None) -> str:
    tag = "" if only is None else f".t{only}"
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + tag + ".o")
    cmd = [_nvcc(), *ARCH, *_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
    if only is not None:
        cmd.append(f"-DALM_INST_ONLY={only}")
    if verbose_ptxas and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "alm.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile every source for sm_103a and link ``libalm_gb300.so``; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    units = _units()
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(lambda u: _compile(u[0], verbose_ptxas, u[1]), units))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
