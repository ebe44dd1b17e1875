"""In-tree build of the CUDA library libpg.so (sm_103a) from csrc/.

The translation units are compiled in parallel by nvcc and linked into
paper_2112_09728_gb300/_lib/libpg.so. The same sources compiled with
PG_BOUNDS_CHECK give libpg_bounds.so, whose kernels check every index that
depends on the data and report a violation through pg_check instead of
accessing memory out of bounds (for tests). No torch is needed to build.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libpg.so")
LIB_BOUNDS = os.path.join(OUT, "libpg_bounds.so")
SOURCES = ["pg_kernels.cu", "pg_reuse.cu", "pg_grad.cu", "pg_api.cu", "pg_params.cu", "pg_noalloc.cu"]
HEADERS = ["pg_device.cuh", "pg_common.cuh", "pg_launch.h", "pg_params.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpg.so")


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(SRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "pg.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, bounds_check: bool | None = None) -> str:
    """Build libpg.so and libpg_bounds.so (bounds_check None), or only the
    one asked for; returns the path of libpg.so (or of the one built)."""
    variants = [False, True] if bounds_check is None else [bool(bounds_check)]
    todo = [v for v in variants if force or _stale(LIB_BOUNDS if v else LIB)]
    if todo:
        _build(todo, verbose)
    return LIB_BOUNDS if bounds_check else LIB


def _build(variants, verbose):
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(job):
        src, checked = job
        obj = os.path.join(OUT, ("bounds_" if checked else "") + src.replace(".cu", ".o"))
        cmd = [cc] + common + (["-DPG_BOUNDS_CHECK"] if checked else []) + ["-c", os.path.join(SRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    jobs = [(src, v) for v in variants for src in SOURCES]
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, log in results:
            print(log)
    for k, v in enumerate(variants):
        lib = LIB_BOUNDS if v else LIB
        objs = [o for o, _ in results[k * len(SOURCES):(k + 1) * len(SOURCES)]]
        tmp = lib + ".tmp%d" % os.getpid()
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
