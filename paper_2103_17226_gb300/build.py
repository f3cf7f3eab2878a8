"""Build the native library in-tree: libqkc.so (CUDA kernels + C-ABI + AC compiler)
for sm_103a.  Objects are compiled in parallel; nothing is installed elsewhere."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libqkc.so"
INCLUDE = ROOT / "include"

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _sources():
    return [CSRC / "qkc.cu", CSRC / "qkc_compile.cpp"]


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> Path:
    """Compile csrc/*.cu and csrc/*.cpp into _build/libqkc.so (skipped when up to date)."""
    BUILD.mkdir(exist_ok=True)
    srcs = _sources()
    deps = srcs + [INCLUDE / "qkc.h", Path(__file__)]
    if not force and not _stale(LIB, deps):
        return LIB
    objs = []
    cmds = []
    for src in srcs:
        obj = BUILD / (src.name + ".o")
        objs.append(obj)
        if src.suffix == ".cu":
            cmds.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)])
        else:
            cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)])
    with ThreadPoolExecutor(len(cmds)) as ex:
        outs = list(ex.map(_run, cmds))
    tmp = BUILD / "libqkc.so.tmp"
    outs.append(_run([NVCC, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]))
    os.replace(tmp, LIB)
    if verbose:
        print("".join(outs))
    return LIB
