"""Builds librx.so (all CUDA kernels and the C-ABI runtime) for sm_103a.

Each translation unit is compiled by its own nvcc process in parallel and
the objects are linked into ``paper_2108_07001_gb300/librx.so``.  Objects
go to ``paper_2108_07001_gb300/_build/``; both are git-ignored.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librx.so")
SOURCES = ["k_peak.cu", "k_cd.cu", "k_mimo.cu", "k_bps.cu", "k_bps2.cu", "k_ber.cu", "k_noalloc.cu", "rx_runtime.cu", "rx_batch.cu",
           "rx_server.cu", "rx_tune.cu", "k_kk.cu", "rx_kk.cu", "k_kkrx.cu", "rx_kkrx.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the receiver library needs the CUDA toolkit")


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link; returns the library path.  Raises on any error."""
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(os.path.dirname(HERE), "include", "rx.h"))
    newest_hdr = max(os.path.getmtime(p) for p in hdrs)
    procs, objs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        op = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(op)
        if (not force and os.path.exists(op)
                and os.path.getmtime(op) >= max(os.path.getmtime(sp), newest_hdr)):
            continue
        cmd = [nv, *ARCH, *FLAGS, "-c", sp, "-o", op]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"--- {src}\n{text}")
        elif verbose and text.strip():
            print(text, flush=True)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nv, *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
