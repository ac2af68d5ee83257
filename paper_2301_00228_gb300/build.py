"""Build the CUDA library liblbps.so in-tree for sm_103a (GB300).

Each .cu file compiles in its own nvcc process (in parallel), then one link
step produces ``paper_2301_00228_gb300/liblbps.so``.  Objects go to
``_build/`` at the repository root.  No GPU is needed to build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = ROOT / "_build"
LIB = PKG / "liblbps.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(outp: Path, deps) -> bool:
    if not outp.exists():
        return True
    t = outp.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> Path:
    """Compile liblbps.so; checked=True builds liblbps_checked.so with every
    kernel memory access range- and alignment-checked (LBPS_CHECKED)."""
    BUILD.mkdir(exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + list(INCLUDE.glob("*.h"))
    # -fmad=false: no compiler-chosen multiply-add contraction, so every kernel
    # that evaluates a shared formula gets the same bits (the hot loops use
    # explicit fused intrinsics where they want them).
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I", str(INCLUDE),
                    "-I", str(CSRC)]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    if checked:
        flags += ["-DLBPS_CHECKED"]
    lib = PKG / ("liblbps_checked.so" if checked else "liblbps.so")
    procs = []
    objs = []
    for src in sources():
        obj = BUILD / (src.stem + ("_checked" if checked else "") + ".o")
        objs.append(obj)
        if force or ptxas_info or _stale(obj, [src] + headers):
            cmd = [nvcc()] + flags + ["-c", str(src), "-o", str(obj)]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out and (verbose or ptxas_info or p.returncode != 0):
            print(out, file=sys.stderr)
        if p.returncode != 0:
            failed.append(src.name)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    if force or procs or _stale(lib, objs):
        tmp = lib.with_suffix(f".so.{os.getpid()}")
        cmd = [nvcc()] + ARCH + ["-shared", "-o", str(tmp)] + [str(o) for o in objs]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    out = build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv)
    print(out)
