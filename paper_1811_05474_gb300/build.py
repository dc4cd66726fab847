"""Compile libmt (the CUDA C-ABI library) for sm_103a, in-tree.

The translation units under ``csrc/`` are compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) and linked into
``_build/libmt.so`` next to this file.  The build is skipped when the
library is newer than every source.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libmt.so"
SOURCES = ["mt_api.cu", "mt_move_sort.cu", "mt_transfer.cu", "mt_io.cu", "mt_noalloc.cu", "mt_fused.cu",
           "mt_tune.cu", "mt_server.cu", "mt_probe.cu"]
HEADERS = [CSRC / "mt_internal.cuh", CSRC / "mt_pair.cuh", ROOT / "include" / "mt.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    found = shutil.which("nvcc")
    if found:
        return found
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _stale(lib: Path, deps) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    deps = [CSRC / s for s in SOURCES] + HEADERS
    if not force and not _stale(LIB, deps):
        return LIB
    obj_dir = BUILD / "obj"
    obj_dir.mkdir(parents=True, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for s in SOURCES:
        o = obj_dir / (Path(s).stem + ".o")
        objs.append(o)
        cmd = [cc, *ARCH, *FLAGS, "-c", str(CSRC / s), "-o", str(o)]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"$ {' '.join(cmd)}\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = BUILD / f"libmt.{os.getpid()}.so"
    cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
