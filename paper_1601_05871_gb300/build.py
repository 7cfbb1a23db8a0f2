"""Builds paper_1601_05871_gb300/_build/libick.so in-tree.

Host C++ (symbolic phase and C ABI) is compiled by g++ with OpenMP, the CUDA kernels by
nvcc for sm_103a only, in parallel; the objects are linked with the static CUDA
runtime.  A rebuild happens only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def lib_path() -> str:
    return os.path.join(BUILD, "libick.so")


def _sources():
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(ROOT, "include", "*.h")))
    return cpp, cu, hdr


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    cpp, cu, hdr = _sources()
    out = lib_path()
    if not force and not _stale(out, cpp + cu + hdr + [__file__]):
        return out
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(CUDA, "include")]
    jobs = []
    objs = []
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        # -ffp-contract=off: the host cost models give the same claim orders on every
        # architecture (no machine-dependent fused multiply-adds)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-Wall",
                     "-Wno-unused-function",
                     *inc, "-c", src, "-o", obj])
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [os.path.join(CUDA, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17",
               "-Xcompiler", "-fPIC", *inc, "-c", src, "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for cmd, log in zip(jobs, logs):
            if log.strip():
                print(os.path.basename(cmd[-3]), log)
    tmp = out + f".tmp{os.getpid()}"
    _run(["g++", "-shared", "-fopenmp", "-o", tmp, *objs, "-L", os.path.join(CUDA, "lib64"),
          "-Wl,-Bstatic", "-lcudart_static", "-Wl,-Bdynamic", "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
