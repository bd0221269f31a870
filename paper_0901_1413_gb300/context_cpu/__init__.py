"""Context baseline: the paper's bitsliced Four-Russians method on the host CPU.

Boothby & Bradshaw measured their CPU implementation (Table 1, a 2.6 GHz
Opteron).  This module runs the same method, written for this project in C
with OpenMP (``m4rm_cpu.c``), on the machine's own cores so that the paper's
numbers, this CPU and the GPU library can be compared at the same sizes.

It is NOT part of the product path: ``fq.matmul`` never calls it and the GPU
library has no CPU fallback.  ``python -m paper_0901_1413_gb300.context_cpu``
prints the comparison at the paper's sizes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "m4rm_cpu.c")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libm4rm_cpu.so")
FIELDS = (2, 3, 4, 5, 7)

_lib = None


def build(force: bool = False) -> str:
    """Compile ``m4rm_cpu.c`` with the host C compiler (plain -O3, OpenMP)."""
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64 = ctypes.c_int64
        lib.fq_cpu_m4rm.argtypes = [ctypes.c_int, i64, i64, i64, u8p, u8p, u8p, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double)]
        lib.fq_cpu_m4rm.restype = ctypes.c_int
        lib.fq_cpu_threads.argtypes = [ctypes.c_int]
        lib.fq_cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads_used(threads: int = 0) -> int:
    return int(_load().fq_cpu_threads(int(threads)))


def default_k(q: int, m: int, threads: int = 0) -> int:
    """Block size balancing each thread's table builds (2^k entries) against its
    lookups (rows x basis size) per block."""
    d = 1 if q == 2 else (2 if q in (3, 4) else 3)
    rows = max(1, m // max(1, threads_used(threads)))
    return int(min(10, max(2, round(math.log2(max(2, rows * d / 2))))))


def matmul(q: int, A: np.ndarray, B: np.ndarray, k: int = 0, threads: int = 0):
    """C = A B by the CPU bitsliced M4RM; returns (C, milliseconds of the
    multiplication on packed planes)."""
    if q not in FIELDS:
        raise ValueError("unsupported field size %r" % (q,))
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    if (A.size and A.max() >= q) or (B.size and B.max() >= q):
        raise ValueError("residue out of range")
    m, l = A.shape
    n = B.shape[1]
    k = k or default_k(q, m, threads)
    C = np.zeros((m, n), dtype=np.uint8)
    ms = ctypes.c_double(0.0)
    p = lambda X: X.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    rc = _load().fq_cpu_m4rm(q, m, l, n, p(A), p(B), p(C), int(k), int(threads), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError("fq_cpu_m4rm failed with status %d" % rc)
    return C, ms.value
