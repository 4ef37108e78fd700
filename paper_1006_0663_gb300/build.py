"""Builds the in-tree CUDA library ``_build/libteuk.so`` for sm_103a with nvcc.

Four translation units are compiled in parallel: the C ABI layer and one unit per
arithmetic (FP64, double-double, quad-double), then linked as one shared library.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libteuk.so")
ROOT = os.path.dirname(HERE)
HEADERS = ["mw.cuh", "mw_func.cuh", "ix.cuh", "ixq.cuh", "teuk_ix.cuh", "teuk_kernels.cuh", "teuk_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources():
    units = [("teuk_capi", "teuk_capi.cu", []), ("teuk_noalloc", "teuk_noalloc.cu", []),
             ("teuk_batch", "teuk_batch.cu", [])]
    for w in (1, 2, 4):
        units.append((f"teuk_w{w}", "teuk_prec.cu", [f"-DTEUK_WORDS={w}"]))
    for w in (2, 4):
        units.append((f"teuk_ixk_w{w}", "teuk_ixk.cu", [f"-DTEUK_WORDS={w}"]))
    return units


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in HEADERS + ["teuk_capi.cu", "teuk_prec.cu", "teuk_noalloc.cu",
                                                          "teuk_batch.cu", "teuk_ixk.cu"]]
    files.append(os.path.join(ROOT, "include", "teuk.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libteuk.so."""
    with _lock:
        os.makedirs(BUILD, exist_ok=True)
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
            return LIB
        nvcc = _nvcc()
        common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                         "-I", CSRC, "-I", os.path.join(ROOT, "include")]
        procs = []
        objs = []
        for name, src, extra in _sources():
            obj = os.path.join(BUILD, f"{name}.o")
            cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common + extra
            if verbose:
                cmd += ["-Xptxas", "-v"]
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        failed = []
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode != 0:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode != 0:
                failed.append(" ".join(cmd))
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
