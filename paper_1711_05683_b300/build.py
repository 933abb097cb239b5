"""Build the in-tree CUDA library ``libhydra_phsp.so`` for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhydra_phsp.so")
SOURCES = [os.path.join(CSRC, "phsp.cu"), os.path.join(CSRC, "phsp_batch.cu"), os.path.join(CSRC, "phsp_batch_f32.cu"),
           os.path.join(CSRC, "phsp_extras.cu"), os.path.join(CSRC, "phsp_vegas.cu"),
           os.path.join(CSRC, "phsp_peaks.cu"), os.path.join(CSRC, "phsp_serve.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhydra_phsp.so")


OBJDIR = os.path.join(PKG, "_build")
# -fmad=false: no implicit contraction; the kernels write every fused multiply-add out, so
# each event's rounding is fixed by the source at every launch shape.
CFLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-fmad=false",
          "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE]


def command(out: str = LIB, extra: list[str] | None = None) -> list[str]:
    """One-step build command (all sources, one nvcc invocation)."""
    return [nvcc(), *CFLAGS, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
            *(extra or []), "-o", out, *SOURCES]


def _compile(src: str, extra) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    subprocess.check_call([nvcc(), *CFLAGS, *(extra or []), "-c", "-o", obj, src])
    return obj


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units in parallel, then link libhydra_phsp.so."""
    if force or needs_build():
        from concurrent.futures import ThreadPoolExecutor
        os.makedirs(OBJDIR, exist_ok=True)
        extra = ["-Xptxas", "-v"] if verbose else None
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda src: _compile(src, extra), SOURCES))
        tmp = LIB + ".tmp"
        subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                               "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
                               "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
