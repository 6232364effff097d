"""Builds the in-tree CUDA library ``_build/liblbm_gb300.so`` for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with the C ABI of ``include/lbm.h``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "liblbm_gb300.so"
SOURCES = ["lbm_api.cu", "lbm_kernels_f32.cu", "lbm_kernels_f64.cu", "lbm_kernels_f16.cu", "lbm_noalloc.cu",
           "lbm_server.cu"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_gb300.so")


def _inputs_newer_than(target: Path) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    deps = list(CSRC.glob("*")) + [ROOT / "include" / "lbm.h", Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    if not force and not _inputs_newer_than(LIB):
        return LIB
    OUT.mkdir(exist_ok=True)
    cc = nvcc()
    common = GENCODE + ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC",
                        "-I", str(ROOT / "include"), "-I", str(CSRC)]
    if verbose_ptxas or os.environ.get("LBM_PTXAS_VERBOSE"):
        common += ["-Xptxas", "-v"]

    def compile_one(src: str) -> tuple[str, str]:
        obj = OUT / (Path(src).stem + ".o")
        cmd = [cc, *common, "-c", str(CSRC / src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return str(obj), r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for _, log in results:
        if log.strip() and (verbose_ptxas or os.environ.get("LBM_PTXAS_VERBOSE")):
            sys.stderr.write(log)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [cc, *GENCODE, "-shared", "-o", str(tmp)] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
