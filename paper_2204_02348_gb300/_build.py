"""Build the native library in-tree: every ``csrc/*.cu`` with nvcc for sm_103a, ``csrc/*.cpp`` with g++,
compiled in parallel and linked into ``_native/libdigholo_gb300.so``; the same CUDA sources compiled again with
``-DDH_CHECKED`` give the bounds-checked library ``_native/libdigholo_gb300_checked.so`` (loaded by the package
when the environment sets DH_CHECKED=1).

Run ``python paper_2204_02348_gb300/_build.py`` (or ``__graft_entry__.build()``).  Set DH_PTXAS_VERBOSE=1 to
print register and shared-memory usage of every kernel.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_native")
LIB = os.path.join(OUT, "libdigholo_gb300.so")
LIB_CHECKED = os.path.join(OUT, "libdigholo_gb300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    deps = cu + cpp + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return cu, cpp, deps


def _up_to_date(deps) -> bool:
    for lib in (LIB, LIB_CHECKED):
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not (all(os.path.getmtime(d) <= t for d in deps) and os.path.getmtime(__file__) <= t):
            return False
    return True


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return cmd, r.returncode, r.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    cu, cpp, deps = _sources()
    if not force and _up_to_date(deps):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    ptxas_v = ["-Xptxas", "-v"] if os.environ.get("DH_PTXAS_VERBOSE") else []
    jobs = []
    objs, objs_checked = [], []
    os.makedirs(os.path.join(OUT, "checked"), exist_ok=True)
    for src in cu:
        for checked in (False, True):
            obj = os.path.join(OUT, "checked" if checked else "", os.path.basename(src) + ".o")
            (objs_checked if checked else objs).append(obj)
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                         *(["-DDH_CHECKED"] if checked else []), *ptxas_v, *inc, "-c", src, "-o", obj])
    for src in cpp:
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        objs.append(obj)
        objs_checked.append(obj)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *inc,
                     "-I", "/usr/local/cuda/include", "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(_run, jobs))
    failed = [(c, o) for c, rc, o in results if rc != 0]
    for c, rc, o in results:
        if verbose or ptxas_v or rc != 0:
            sys.stderr.write(" ".join(c) + "\n" + o)
    if failed:
        raise RuntimeError("native build failed:\n" + "\n".join(o for _, o in failed))
    for lib, o_list in ((LIB, objs), (LIB_CHECKED, objs_checked)):
        tmp = lib + ".tmp"
        cmd, rc, o = _run([nvcc, *ARCH, "-shared", "-o", tmp, *o_list, "-lpthread"])
        if rc != 0:
            raise RuntimeError("link failed:\n" + o)
        os.replace(tmp, lib)
    return LIB

if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
