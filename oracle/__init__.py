"""CPU oracle for the GPU-sharing hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never loads it,
and it shares no code with the CUDA path: the compute lives in
``gvm_oracle.c`` (plain C, binary64 matrix multiply), compiled with gcc.

What it defines (the paper is Li, Narayana and El-Ghazawi, "Efficient
Resource Sharing Through GPU Virtualization on Accelerated High Performance
Computing Systems"):

* ``vadd`` -- the vector-addition task of Table 2: one binary32 addition per
  element.
* ``vmul`` -- the vector-multiplication task of Table 2 (VecMult): ``iters``
  binary32 multiplications by ``b`` per element, each rounded.
* ``sgemm64`` -- the single-precision matrix-multiplication task of Table 2
  (Section 6), as the exact product computed in binary64.
* ``run_rank`` / ``run_workload`` -- every rank's tasks in its submission
  order, each in isolation: sharing a GPU through the virtualization manager
  changes only timing (Section 4.2.2, Section 5), so a task's result depends
  on its own inputs alone.
* ``model`` -- the execution-model closed forms, Eqs. 1-11 (Section 4).

Pins (``tests/test_oracle.py``): numpy float32 addition and float64 matmul,
hand-checked IEEE cases, integer-valued products that are exact, identity,
zero and outer-product cases, brute force with exact rationals, and the
limits and special cases the model equations must satisfy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import model  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gvm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ``gvm_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            f32p = ctypes.POINTER(ctypes.c_float)
            f64p = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_vadd_f32.argtypes = [f32p, f32p, f32p, i64]
            lib.oracle_vadd_f32.restype = None
            lib.oracle_vmul_f32.argtypes = [f32p, f32p, f32p, i64, ctypes.c_int32]
            lib.oracle_vmul_f32.restype = None
            lib.oracle_sgemm_f64.argtypes = [f32p, f32p, f64p, i64, i64, i64]
            lib.oracle_sgemm_f64.restype = None
            lib.oracle_rel_fro_err.argtypes = [f32p, f64p, i64]
            lib.oracle_rel_fro_err.restype = ctypes.c_double
            _lib = lib
    return _lib


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _ptr(x, ct):
    return x.ctypes.data_as(ctypes.POINTER(ct))


def vadd(a, b) -> np.ndarray:
    """c = a + b in binary32 (Table 2, VecAdd)."""
    a, b = _f32(a), _f32(b)
    if a.shape != b.shape:
        raise ValueError("vadd operands differ in shape")
    c = np.empty_like(a)
    _load().oracle_vadd_f32(_ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float),
                            _ptr(c, ctypes.c_float), a.size)
    return c


def vmul(a, b, iters: int) -> np.ndarray:
    """c = a * b * ... * b with ``iters`` binary32 products (Table 2, VecMult)."""
    a, b = _f32(a), _f32(b)
    if a.shape != b.shape:
        raise ValueError("vmul operands differ in shape")
    if not 1 <= iters <= 1024:
        raise ValueError("vmul iters outside 1..1024")
    c = np.empty_like(a)
    _load().oracle_vmul_f32(_ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float),
                            _ptr(c, ctypes.c_float), a.size, iters)
    return c


def sgemm64(A, B) -> np.ndarray:
    """C = A @ B in binary64 from binary32 row-major operands (Table 2, MM)."""
    A, B = _f32(A), _f32(B)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError(f"sgemm64 shapes {A.shape} x {B.shape}")
    M, K = A.shape
    N = B.shape[1]
    C = np.empty((M, N), dtype=np.float64)
    _load().oracle_sgemm_f64(_ptr(A, ctypes.c_float), _ptr(B, ctypes.c_float),
                             _ptr(C, ctypes.c_double), M, N, K)
    return C


def rel_fro_err(C, R) -> float:
    """||C - R||_F / ||R||_F with binary64 norms (the SGEMM parity metric)."""
    C = _f32(C)
    R = np.ascontiguousarray(R, dtype=np.float64)
    if C.size != R.size:
        raise ValueError("rel_fro_err size mismatch")
    return float(_load().oracle_rel_fro_err(_ptr(C, ctypes.c_float), _ptr(R, ctypes.c_double), C.size))


def run_task(spec):
    """Result of one task spec (see ``synth.TaskSpec``) computed alone."""
    import synth

    if spec.kind == synth.TASK_VADD:
        a, b = synth.vadd_inputs(spec.seed, spec.n)
        return vadd(a, b)
    if spec.kind == synth.TASK_VMUL:
        a, b = synth.vmul_inputs(spec.seed, spec.n)
        return vmul(a, b, spec.k)
    if spec.kind == synth.TASK_SGEMM:
        A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
        return sgemm64(A, B)
    raise ValueError(f"unknown task kind {spec.kind}")


def run_rank(specs):
    """One rank's tasks in submission order, each in isolation."""
    return [run_task(s) for s in sorted(specs, key=lambda s: s.index)]


def run_workload(workload, threads: int | None = None):
    """Every rank's tasks, one rank per thread; returns {(rank, index): result}."""
    ranks = workload.by_rank()
    workers = threads or min(len(ranks), os.cpu_count() or 1)
    out = {}
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        for r, res in zip(range(len(ranks)), ex.map(run_rank, ranks)):
            for spec, val in zip(ranks[r], res):
                out[(r, spec.index)] = val
    return out
