"""Build the CUDA library libadft.so in-tree for sm_103a with nvcc.

Translation units are compiled in parallel, then linked into
paper_2406_11185_gb300/lib/libadft.so.  Nothing is installed outside the tree.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
OUT = os.path.join(OUT_DIR, "libadft.so")
# The units are ordered longest compile first (the FP32 d-class units), so the
# parallel build finishes about when its longest unit does.
SOURCES = ["adft_eri32_j.cu", "adft_eri32_i.cu", "adft_eri32_e.cu"] + [
    f"adft_eri{p}_{g}.cu" for p in ("64", "32") for g in ("a", "b", "c", "d", "e", "f", "g", "h")
    if f"adft_eri{p}_{g}.cu" != "adft_eri32_e.cu"] + [
    "adft_core.cu", "adft_dispatch.cu", "adft_grad.cu", "adft_static.cu", "adft_peaks.cu", "adft_onee.cu"] + [
    f"adft_grad{p}_{g}.cu" for p in ("64", "32") for g in ("a", "b", "c")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
            "-I", CSRC]


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.join(OUT_DIR, "obj"), exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "adft.h"))
    procs, objs = [], []
    t0 = time.time()
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, "obj", src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc(), *_flags(), "-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), o, src))
    for p, o, src in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
            raise RuntimeError(f"nvcc failed on {src}")
        os.replace(o + ".tmp", o)
    if force or procs or not os.path.exists(OUT):
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", OUT + ".tmp", *objs, "-lcudart"])
        os.replace(OUT + ".tmp", OUT)
    if verbose:
        print(f"libadft.so ready in {time.time() - t0:.1f} s", flush=True)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
