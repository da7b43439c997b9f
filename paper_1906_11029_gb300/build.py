"""Build the in-tree C-ABI library ``_lib/libmtp.so`` for sm_103a.

Host C++ (mesh, pitcher, reference tables) is compiled with g++ and
``-ffp-contract=off`` so the pitcher's FP64 arithmetic is exactly as specified;
the CUDA translation units are compiled in parallel with one ``-gencode`` for
sm_103a and linked with the static CUDA runtime.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmtp.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SOURCES = ["mtp_host.cpp", "mtp_tables.cpp"]
CU_SOURCES = ["mtp_cuda.cu", "mtp_k64.cu", "mtp_k32.cu", "mtp_ks.cu", "mtp_krk.cu", "mtp_kv.cu", "mtp_kv2.cu", "mtp_ktc5.cu", "mtp_ktc.cu", "mtp_kb.cu", "mtp_adj.cu", "mtp_probe.cu", "mtp_noalloc.cu", "mtp_pitch.cu"]
HEADERS = ["mtp_internal.h", "mtp_kernels.cuh", "mtp_adjoint.cuh", "mtp_launch.cuh", "../../include/mtp.h"]


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(BUILD, "ARCH")
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch:
        force = True                      # objects from another machine are never reused
    headers = [os.path.join(CSRC, h) for h in HEADERS]
    inc = ["-I", os.path.join(HERE, "..", "include"), "-I", CSRC]
    jobs, objs = [], []
    cxx = shutil.which("g++") or "g++"
    for s in CXX_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _newer([src] + headers, obj):
            jobs.append([cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
                         *inc, "-I", os.path.join(CUDA_HOME, "include"), "-c", src, "-o", obj])
    for s in CU_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _newer([src] + headers, obj):
            cmd = [NVCC, *GENCODE, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                   *inc, "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    log = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(_run, jobs):
            log.append(out)
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([NVCC, *GENCODE, "-shared", "-cudart", "static", "-Xcompiler", "-fPIC", *objs, "-o", tmp])
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(arch)
    text = "\n".join(x for x in log if x.strip())
    if verbose and text:
        print(text)
    return text


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
