"""Builds the package's native libraries in-tree.

* ``libte.so``    -- the C-ABI TE iteration library (CUDA, sm_103a only).
* ``libtegen.so`` -- the seeded instance generator's k-shortest-path helper
  (host C++ with OpenMP).

Both are compiled next to their sources so that the built files travel with
the source tree.  ``python -m paper_2605_01748_b300.build`` builds both.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG_DIR, "csrc")
REPO = os.path.dirname(PKG_DIR)
INCLUDE = os.path.join(REPO, "include")

LIBTE = os.path.join(PKG_DIR, "libte.so")
LIBTEGEN = os.path.join(PKG_DIR, "libtegen.so")

TE_SOURCES = ["te_api.cu", "te_layout.cu", "te_iter.cu", "te_batch.cu", "te_adjoint.cu", "te_proj.cu", "te_gap.cu",
              "te_literal.cu",
              "te_noalloc.cu"]
GEN_SOURCES = [os.path.join("gen", "kpaths.cpp")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libte.so")


def _stale(target: str, sources: list[str], extra: list[str] = ()) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, s) for s in sources] + list(extra)
    for d in deps:
        if os.path.exists(d) and os.path.getmtime(d) > t:
            return True
    return False


def _headers() -> list[str]:
    out = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out


def build_gen(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale(LIBTEGEN, GEN_SOURCES):
        return LIBTEGEN
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", LIBTEGEN]
    cmd += [os.path.join(CSRC, s) for s in GEN_SOURCES]
    _run(cmd, verbose)
    return LIBTEGEN


def build_te(force: bool = False, verbose: bool = False, out: str = LIBTE) -> str:
    if not force and not _stale(out, TE_SOURCES, _headers()):
        return out
    nvcc = _nvcc()
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, "-o", out]
    if os.environ.get("TE_PTXAS_VERBOSE"):
        cmd += ["-Xptxas", "-v"]
    if os.environ.get("TE_ITER_THREADS"):
        cmd += [f"-DTE_ITER_THREADS={int(os.environ['TE_ITER_THREADS'])}"]
    if os.environ.get("TE_ITER_STAGE_ROWS"):
        cmd += [f"-DTE_ITER_STAGE_ROWS={int(os.environ['TE_ITER_STAGE_ROWS'])}"]
    cmd += [os.path.join(CSRC, s) for s in TE_SOURCES]
    cmd += ["-lcudart"]
    _run(cmd, verbose)
    return out


def build_all(force: bool = False, verbose: bool = False) -> None:
    build_gen(force, verbose)
    build_te(force, verbose)


def _run(cmd: list[str], verbose: bool) -> None:
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or res.returncode != 0:
        sys.stdout.write(res.stdout)
        sys.stderr.write(res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"build failed ({res.returncode}): {' '.join(cmd)}")


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose=True)
