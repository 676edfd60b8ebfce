"""Builds libkselect.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Every .cu file under csrc/ is one translation unit; simt_shard.cu is compiled
once per shard (-DKS_SHARD=i).  Objects compile in parallel and are linked
with the shared CUDA runtime (the one PyTorch also loads).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkselect.so")
# Debug variant: every global access of the FP32 kernels checked against the
# operands' extents (KS_DEBUG_BOUNDS), over every DEBUG_SUBSET-th SIMT config.
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "libkselect_debug.so")
DEBUG_SUBSET = 7
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
N_SHARDS = 12
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags() -> list[str]:
    return ["-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
            "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _units(build_dir: str) -> list[tuple[str, str, list[str]]]:
    units = []
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith(".cu"):
            continue
        src = os.path.join(CSRC, name)
        if name == "simt_shard.cu":
            for i in range(N_SHARDS):
                units.append((src, os.path.join(build_dir, f"simt_shard_{i}.o"), [f"-DKS_SHARD={i}"]))
        else:
            units.append((src, os.path.join(build_dir, name[:-3] + ".o"), []))
    return units


def _digest(paths: list[str], extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()


def build_library(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile (if sources changed) and link libkselect.so; returns its path."""
    return _build(BUILD, LIB, [], force, jobs, verbose)


def build_debug_library(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """The bounds-checking debug variant (libkselect_debug.so, same C ABI, a
    subset of the FP32 configs); returns its path."""
    return _build(DEBUG_BUILD, DEBUG_LIB, ["-DKS_DEBUG_BOUNDS", f"-DKS_SUBSET={DEBUG_SUBSET}"], force, jobs,
                  verbose)


def _build(build_dir: str, lib: str, defines: list[str], force: bool, jobs: int | None, verbose: bool) -> str:
    os.makedirs(build_dir, exist_ok=True)
    srcs = [os.path.join(CSRC, n) for n in os.listdir(CSRC) if n.endswith((".cu", ".cuh", ".h"))]
    srcs.append(os.path.join(INCLUDE, "kselect.h"))
    stamp_path = os.path.join(build_dir, "stamp")
    digest = _digest(srcs, " ".join(_flags() + defines) + os.uname().machine)
    if not force and os.path.exists(lib) and os.path.exists(stamp_path):
        if open(stamp_path).read() == digest:
            return lib
    cc = nvcc()
    units = [(src, obj, extra + defines) for src, obj, extra in _units(build_dir)]
    jobs = jobs or max(1, os.cpu_count() or 1)

    def compile_one(u):
        src, obj, extra = u
        cmd = [cc, *_flags(), *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {extra}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(jobs) as ex:
        for msg in ex.map(compile_one, units):
            if verbose and msg.strip():
                sys.stderr.write(msg)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [cc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[u[1] for u in units]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_path, "w") as f:
        f.write(digest)
    return lib


if __name__ == "__main__":
    t = __import__("time").time()
    print(build_library(force="--force" in sys.argv, verbose=True), f"{__import__('time').time() - t:.1f}s")
