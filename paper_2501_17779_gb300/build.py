"""Compile libfftalign.so (the CUDA kernels and the C ABI) for sm_103a, in-tree.

Each translation unit is compiled by nvcc in parallel and the objects are
linked into paper_2501_17779_gb300/_build/libfftalign.so (static CUDA
runtime).  nvcc cross-compiles without a GPU, so this also runs on a CPU-only
host.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libfftalign.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", str(INCLUDE), "-I", str(CSRC)]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if Path(cand).exists() else "nvcc"


def sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu"))


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = sources() + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


PEAK_SRC = CSRC / "probe" / "fp64_peak.cu"
PEAK_LIB = OUT_DIR / "libfapeak.so"


def build_probe(force: bool = False) -> Path:
    """The FP64 peak probe used by bench.py (separate from the alignment ABI)."""
    if not force and PEAK_LIB.exists() and PEAK_LIB.stat().st_mtime >= PEAK_SRC.stat().st_mtime:
        return PEAK_LIB
    OUT_DIR.mkdir(exist_ok=True)
    tmp = OUT_DIR / f"libfapeak.so.{os.getpid()}"
    subprocess.run([_nvcc(), *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", "-o", str(tmp),
                    str(PEAK_SRC)], check=True)
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not _stale():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()

    def compile_one(src: Path) -> Path:
        obj = OUT_DIR / (src.stem + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", str(src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs) + 1)) as ex:
        probe = ex.submit(build_probe, force)
        objs = list(ex.map(compile_one, srcs))
        probe.result()
    tmp = OUT_DIR / f"libfftalign.so.{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
