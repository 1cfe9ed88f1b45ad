"""Build step of the CUDA library: nvcc for sm_103a, one object per source
compiled in parallel, linked into paper_0802_0748_gb300/_build/libscocg.so."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libscocg.so"
SOURCES = ["api.cu", "layout.cu", "solver.cu", "solver_resume.cu", "hubbard.cu", "adjoint.cu", "noalloc.cu", "multi.cu", "block.cu",
           "density.cu", "ground.cu", "hubbard2.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include")]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _inputs() -> list[Path]:
    files = [CSRC / s for s in SOURCES]
    files += sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + [ROOT / "include" / "scocg.h"]
    return files


def lib_path(checked: bool = False, variant: str = "") -> Path:
    if variant:
        return BUILD / variant / "libscocg.so"
    return BUILD / "checked" / "libscocg.so" if checked else LIB


def up_to_date(checked: bool = False, variant: str = "") -> bool:
    lib = lib_path(checked, variant)
    if not lib.exists():
        return False
    t = lib.stat().st_mtime
    return all(f.stat().st_mtime <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False, variant: str = "",
          defines: tuple = ()) -> Path:
    """Compile every CUDA source for sm_103a and link the shared library.

    checked=True builds the bounds-checked variant (-DSCOCG_CHECKED) into
    _build/checked/: every data-dependent index is tested and a bad one is
    reported by the solve instead of being used.  variant/defines build other
    instrumented variants (e.g. -DSCOCG_PHASE_TIMERS) into _build/<variant>/."""
    lib = lib_path(checked, variant)
    if not force and up_to_date(checked, variant):
        return lib
    obj_dir = lib.parent / "obj"
    obj_dir.mkdir(parents=True, exist_ok=True)
    nvcc = _nvcc()
    extra = (["-DSCOCG_CHECKED"] if checked else []) + [f"-D{d}" for d in defines]

    def compile_one(src: str) -> Path:
        out = obj_dir / (Path(src).stem + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", str(CSRC / src), "-o", str(out)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return out

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib.with_suffix(f".{os.getpid()}.tmp")
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *map(str, objs), "-o", str(tmp)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
