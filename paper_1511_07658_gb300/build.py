"""In-tree build of libgvm.so for sm_103a (GB300).

Each .cu file compiles in its own nvcc process (in parallel), then one link
step produces ``paper_1511_07658_gb300/_build/libgvm.so``. The CUDA runtime is
linked statically and the driver is reached through runtime entry points, so
the library loads on a machine without a GPU driver (its calls then return
GVM_ENODEV).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgvm.so")
SOURCES = ["gvm_host.cu", "gvm_sched.cu", "gvm_kernels.cu", "gvm_noalloc.cu", "gvm_spmd.cu", "gvm_ipc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = [
    "-O3",
    "-std=c++17",
    "-lineinfo",
    "-Xcompiler",
    "-fPIC",
    "-Xcompiler",
    "-fvisibility=hidden",
    "-ftz=false",
    "-prec-div=true",
    "-prec-sqrt=true",
    "-fmad=true",
    "--expt-relaxed-constexpr",
]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps += [os.path.join(ROOT, "include", f) for f in ("gvm.h", "gvm_ipc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


PLAIN_SRC = os.path.join(CSRC, "gvm_plain_rank.c")
PLAIN_EXE = os.path.join(OUT_DIR, "gvm_plain_rank")


def build_plain(force: bool = False) -> str:
    """The plain-form rank program (one process and context per rank), a C
    client of libgvm.so and the CUDA runtime, built with gcc."""
    if not force and os.path.exists(PLAIN_EXE) and os.path.getmtime(PLAIN_EXE) >= max(
            os.path.getmtime(PLAIN_SRC), os.path.getmtime(LIB)):
        return PLAIN_EXE
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    tmp = PLAIN_EXE + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(cuda, "include"), PLAIN_SRC, "-o", tmp, "-L", OUT_DIR, "-lgvm",
           "-Wl,-rpath," + OUT_DIR, "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("gcc failed for the plain-form rank program")
    os.replace(tmp, PLAIN_EXE)
    return PLAIN_EXE


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, s):
            cmd = [nvcc(), *ARCH, *FLAGS, *inc, "-c", s, "-o", o]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose or ptxas_info or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if jobs or force or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    build_plain(force)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
