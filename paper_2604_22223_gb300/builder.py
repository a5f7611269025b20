"""Build libqa.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel to _build/*.o and
linked into paper_2604_22223_gb300/libqa.so with a static CUDA runtime.  A
stamp of the sources, flags and machine architecture makes repeated calls
no-ops; set QA_FORCE_BUILD=1 to rebuild.
"""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqa.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3",
                  "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqa")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp", ".h", ".cuh")))


def _stamp() -> str:
    h = hashlib.sha256()
    for f in _sources() + [os.path.join(ROOT, "include", "qa.h")]:
        with open(f, "rb") as fh:
            h.update(f.encode() + fh.read())
    h.update(" ".join(CUFLAGS + CXXFLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(verbose: bool = False) -> str:
    """Compile every CUDA/C++ source for sm_103a and link libqa.so; returns its path."""
    stamp_file = os.path.join(BUILD, "stamp")
    stamp = _stamp()
    if (os.path.exists(LIB) and os.path.exists(stamp_file) and not os.environ.get("QA_FORCE_BUILD")
            and open(stamp_file).read() == stamp):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
    jobs = []
    for src in _sources():
        if not src.endswith((".cu", ".cpp")):
            continue
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc] + CUFLAGS + ["-c", src, "-o", obj]
        else:
            cmd = ["g++"] + CXXFLAGS + ["-I" + cuda_inc, "-c", src, "-o", obj]
        jobs.append((cmd, obj))

    def run(job):
        cmd, obj = job
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
        if verbose and (p.stdout or p.stderr):
            print(p.stdout + p.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB


# The translation units whose index-map gathers (the -R map and the pair-basis
# term lists) carry bounds checks when compiled with QA_CHECK_BOUNDS.
CHECKED_UNITS = ("qa_fft.cu", "qa_reduced.cu")
LIB_CHECKED = os.path.join(PKG, "libqa_checked.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")


def build_checked(verbose: bool = False) -> str:
    """libqa_checked.so: libqa.so with CHECKED_UNITS recompiled with -DQA_CHECK_BOUNDS
    (an out-of-range gather index then reports QA_EBOUNDS instead of reading out of
    bounds).  A diagnostic build for tests; the product library is libqa.so."""
    build(verbose)
    stamp_file = os.path.join(BUILD_CHECKED, "stamp")
    stamp = _stamp() + "checked"
    if os.path.exists(LIB_CHECKED) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB_CHECKED
    os.makedirs(BUILD_CHECKED, exist_ok=True)
    nvcc = _nvcc()
    objs, jobs = [], []
    for src in _sources():
        if not src.endswith((".cu", ".cpp")):
            continue
        name = os.path.basename(src)
        if name in CHECKED_UNITS:
            obj = os.path.join(BUILD_CHECKED, name + ".o")
            jobs.append([nvcc] + CUFLAGS + ["-DQA_CHECK_BOUNDS", "-c", src, "-o", obj])
            objs.append(obj)
        else:
            objs.append(os.path.join(BUILD, name + ".o"))

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB_CHECKED + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    os.replace(tmp, LIB_CHECKED)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB_CHECKED


if __name__ == "__main__":
    print(build(verbose=True))
