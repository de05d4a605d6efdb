"""Build the CDI CUDA library ``_lib/libcdi.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library with a plain C ABI (include/cdi.h).  ``checked=True`` builds the
bounds-checked variant ``_lib/libcdi_checked.so`` (-DCDI_CHECKED: kernels test
the indices they derive and record bad ones in the device status words).
Usage::

    python -m paper_1803_01262_gb300.build [--force] [--ptxas-v] [--checked]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libcdi.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libcdi_checked.so")
SOURCES = ["cdi_fwd.cu", "cdi_fwd_tma.cu", "cdi_fwd_tb.cu", "cdi_adj.cu", "cdi_batch.cu", "cdi_api.cu",
           "cdi_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The step kernels (single grid, batch, adjoint) flush FP32 denormals (values
# below 1.2e-38) to zero; this removes denormal handling around rsqrtf and is far
# below every tolerance (the adjoint's normal floor is (8 eps)^2 ~ 2e-13).
PER_FILE = {"cdi_fwd.cu": ["-ftz=true"], "cdi_fwd_tma.cu": ["-ftz=true"], "cdi_fwd_tb.cu": ["-ftz=true"],
            "cdi_batch.cu": ["-ftz=true"], "cdi_adj.cu": ["-ftz=true"]}
# No contraction of a product and a sum into a fused multiply-add beyond the fma()
# calls the sources write: the compiler's choice differs between the places an
# expression is inlined (a work unit's prologue and the steady plane loop, one
# tile shape and another), so with contraction the same cell came out one unit
# in the last place apart under different tiles and work splits; without it every
# configuration computes the same bits (and runs as fast).  The adjoint, whose
# configurations promise no such agreement, keeps contraction (4% faster with it).
CONTRACT = {"cdi_adj.cu"}
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
         "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CDI library needs the CUDA toolkit")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "cdi.h"))
    return [f for f in files if os.path.isfile(f)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, ptxas_verbose: bool = False, verbose: bool = False,
          checked: bool = False) -> str:
    """Compile and link the library (the checked variant with ``checked``) if any source
    is newer than it; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    obj_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    missing = [s for s in SOURCES if not os.path.exists(os.path.join(CSRC, s))]
    if missing:
        raise RuntimeError(f"CUDA sources missing: {', '.join(missing)}")
    srcs = SOURCES
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    defs = ["-DCDI_CHECKED"] if checked else []

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        fmad = "-fmad=true" if src in CONTRACT else "-fmad=false"
        cmd = [cc, *ARCH, *FLAGS, fmad, *defs, *PER_FILE.get(src, []), *extra, "-c", os.path.join(CSRC, src),
               "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    for src, _, r in results:
        if verbose or ptxas_verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {src}")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for _, o, _ in results], "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    ap.add_argument("--checked", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas_verbose=a.ptxas_v, verbose=True, checked=a.checked))
