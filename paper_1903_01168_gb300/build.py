"""Build the CUDA library in-tree with nvcc for sm_103a (GB300).

    python -m paper_1903_01168_gb300.build [--force] [--verbose]

Produces ``paper_1903_01168_gb300/_native/liblbm_gb300.so`` (or the path in the
environment variable LBM_GB300_LIB, which the binding then loads) from
``paper_1903_01168_gb300/csrc/*.cu`` and ``include/lbm.h``.  Each translation unit
is compiled to an object in parallel (the step kernels of each storage type sit in
their own units), then the objects are linked.  Rebuilds only when a source is
newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_native")
LIB = os.environ.get("LBM_GB300_LIB") or os.path.join(OUT_DIR, "liblbm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "lbm.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps())


def compile_command(src: str, obj: str, extra: list[str] | None = None) -> list[str]:
    """nvcc command for one unit; LBM_NVCC_FLAGS adds flags (e.g. -DLBM_FUSED_NSLOT=3)."""
    env = os.environ.get("LBM_NVCC_FLAGS", "").split()
    return [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
            *env, *(extra or []), "-c", "-o", obj, src]


def link_command(objs: list[str], out: str) -> list[str]:
    return [nvcc(), *ARCH, "-shared", "-o", out, *objs]


def _run(cmd: list[str]) -> subprocess.CompletedProcess:
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if needed and return its path."""
    if not force and not stale():
        return LIB
    obj_dir = os.path.join(os.path.dirname(LIB), "obj")
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose else []
    srcs = sources()
    tag = f".{os.getpid()}"
    objs = [os.path.join(obj_dir, os.path.basename(p)[:-3] + tag + ".o") for p in srcs]
    cmds = [compile_command(p, o, extra) for p, o in zip(srcs, objs)]
    with ThreadPoolExecutor(max_workers=min(len(cmds), max(1, os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run, cmds))
    for cmd, res in zip(cmds, results):
        if res.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
        if verbose:
            sys.stderr.write(res.stdout + res.stderr)
    tmp = LIB + tag + ".tmp"
    res = _run(link_command(objs, tmp))
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    p = build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(p)
