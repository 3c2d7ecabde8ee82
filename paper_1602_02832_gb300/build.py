"""Builds libhh.so in-tree: nvcc for the CUDA translation units (sm_103a only),
g++ for the host tree builder, compiled in parallel and linked with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhh.so")
PEAKS_LIB = os.path.join(HERE, "libhh_peaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["hh_api.cu", "hh_static.cu", "hh_batch.cu", "hh_gtree.cu"]
CPP = ["hh_tree.cpp"]
HEADERS = ["hh_internal.h", "hh_kernels.cuh", "hh_ctx.h"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP + HEADERS] + [os.path.join(HERE, "..", "include", "hh.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAKS_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    return all(os.path.getmtime(s) <= t for s in _sources() + [os.path.join(CSRC, "hh_peaks.cu")])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v" if verbose else "-O3",
                     "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off,-O2", "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CPP:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-c",
                     os.path.join(CSRC, f), "-o", obj])

    peaks_tmp = PEAKS_LIB + f".tmp{os.getpid()}"
    jobs.append([nvcc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                 os.path.join(CSRC, "hh_peaks.cu"), "-o", peaks_tmp])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    try:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            logs = list(ex.map(run, jobs))
    except Exception:
        if os.path.exists(peaks_tmp):
            os.remove(peaks_tmp)
        raise
    if verbose:
        for lg in logs:
            sys.stderr.write(lg)
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    os.replace(peaks_tmp, PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
