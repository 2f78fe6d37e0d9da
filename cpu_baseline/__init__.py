"""The paper's CPU design (Algorithm 1 with the prefix threads of Section 3.1),
written fresh in C, as a timing baseline on the host cores.

Not a parity reference and not part of the GPU path: only bench.py's CPU
baseline leg loads it.  ``walk(Q, m, prefixes)`` walks the listed prefixes of
the top m variables and returns (min walk value, natural index, threads).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_gray.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcpugray.so")

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = [os.environ.get("CC", "gcc"), "-O3", "-std=c11", "-fPIC", "-shared", "-pthread",
           SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.cg_walk_prefixes.restype = ctypes.c_int
        lib.cg_walk_prefixes.argtypes = [P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                         P(ctypes.c_uint64), ctypes.c_uint64, ctypes.c_int,
                                         P(ctypes.c_double), P(ctypes.c_uint64)]
        _lib = lib
    return _lib


def walk(Q, m: int, prefixes, threads: int = 0):
    """Gray-walk every listed prefix (values of the top m variables)."""
    lib = _load()
    Qd = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    n = Qd.shape[0]
    pre = np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint64))
    best = ctypes.c_double()
    arg = ctypes.c_uint64()
    T = lib.cg_walk_prefixes(Qd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, m,
                             pre.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), pre.shape[0],
                             threads, ctypes.byref(best), ctypes.byref(arg))
    if T < 0:
        raise ValueError("cpu_gray: bad arguments")
    return best.value, int(arg.value), T
