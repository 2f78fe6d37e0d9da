"""CPU oracle for exhaustive QUBO minimisation (arXiv 2310.19373).

TEST INFRASTRUCTURE ONLY.  This package is the correctness reference for the
GPU library.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and never imports it.

Everything here enumerates x in natural binary order (x_i = bit i of idx, the
naive method of Section 3) and evaluates Eq. 1, f(x) = x^T Q x, from scratch
for every state -- no Gray code, no incremental update.  Floating-point Q is
evaluated in FP64 in the canonical order documented in ``qubo_oracle.c``;
integer Q in exact int64.  Ties go to the lowest index.

Functions
---------
evaluate(Q, idx)          f at one state (or an array of states)
brute_min(Q, lo, hi)      (min f, lowest argmin idx) over idx in [lo, hi)
brute_topk(Q, k, lo, hi)  k smallest (value, idx) pairs, lexicographic
blocked_topk(Q, k, lo, hi) brute_topk's answer by the blocked walk (n up to 62)
blocked_min(Q, lo, hi)    brute_min's answer by the blocked walk
segment_minima(Q, seg, nseg, lo)  per-segment minima by the blocked walk
logz(Q, betas)            log sum_x exp(-beta f(x)) and E_beta[x x^T] (FP64)
ising_from_qubo(Q)        the textbook QUBO -> Ising change of variables
ising_energy(J, h, c, s)  energy of spins s in {-1,+1}^n
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        c_dp = ctypes.POINTER(ctypes.c_double)
        c_ip = ctypes.POINTER(ctypes.c_int64)
        c_up = ctypes.POINTER(ctypes.c_uint64)
        lib.orc_eval_f64.restype = ctypes.c_double
        lib.orc_eval_f64.argtypes = [c_dp, ctypes.c_int, ctypes.c_uint64]
        lib.orc_eval_i64.restype = ctypes.c_int64
        lib.orc_eval_i64.argtypes = [c_ip, ctypes.c_int, ctypes.c_uint64]
        lib.orc_eval_many_f64.restype = None
        lib.orc_eval_many_f64.argtypes = [c_dp, ctypes.c_int, c_up, ctypes.c_int64, c_dp]
        lib.orc_eval_many_i64.restype = None
        lib.orc_eval_many_i64.argtypes = [c_ip, ctypes.c_int, c_up, ctypes.c_int64, c_ip]
        lib.orc_min_f64.restype = ctypes.c_int
        lib.orc_min_f64.argtypes = [c_dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int, c_dp, c_up]
        lib.orc_min_i64.restype = ctypes.c_int
        lib.orc_min_i64.argtypes = [c_ip, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int, c_ip, c_up]
        lib.orc_topk_f64.restype = ctypes.c_int
        lib.orc_topk_f64.argtypes = [c_dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, c_dp, c_up]
        lib.orc_topk_i64.restype = ctypes.c_int
        lib.orc_topk_i64.argtypes = [c_ip, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, c_ip, c_up]
        lib.orc_logz_f64.restype = ctypes.c_int
        lib.orc_logz_f64.argtypes = [c_dp, ctypes.c_int, c_dp, ctypes.c_int, ctypes.c_int,
                                     c_dp, c_dp, c_dp, c_up]
        c_u64 = ctypes.c_uint64
        lib.orc_topk_blocked_f64.restype = ctypes.c_int
        lib.orc_topk_blocked_f64.argtypes = [c_dp, ctypes.c_int, c_u64, c_u64, ctypes.c_int,
                                             ctypes.c_int, c_dp, c_up, c_up]
        lib.orc_topk_blocked_i64.restype = ctypes.c_int
        lib.orc_topk_blocked_i64.argtypes = [c_ip, ctypes.c_int, c_u64, c_u64, ctypes.c_int,
                                             ctypes.c_int, c_ip, c_up]
        lib.orc_segmin_blocked_f64.restype = ctypes.c_int
        lib.orc_segmin_blocked_f64.argtypes = [c_dp, ctypes.c_int, c_u64, c_u64, c_u64,
                                               ctypes.c_int, c_dp, c_up]
        lib.orc_segmin_blocked_i64.restype = ctypes.c_int
        lib.orc_segmin_blocked_i64.argtypes = [c_ip, ctypes.c_int, c_u64, c_u64, c_u64,
                                               ctypes.c_int, c_ip, c_up]
        lib.orc_default_threads.restype = ctypes.c_int
        lib.orc_default_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as_matrix(Q):
    """Return (array, is_int): float Q -> contiguous float64, integer Q -> int64."""
    Q = np.asarray(Q)
    if Q.ndim != 2 or Q.shape[0] != Q.shape[1]:
        raise ValueError("Q must be a square matrix")
    if np.issubdtype(Q.dtype, np.integer) or Q.dtype == np.bool_:
        return np.ascontiguousarray(Q, dtype=np.int64), True
    Qd = np.ascontiguousarray(Q, dtype=np.float64)
    if not np.all(np.isfinite(Qd)):
        raise ValueError("Q has non-finite entries")
    return Qd, False


def threads_default() -> int:
    return int(_load().orc_default_threads())


def evaluate(Q, idx):
    """f(x) for x = bits of idx (scalar or array of uint64), Eq. 1."""
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    n = Qm.shape[0]
    scalar = np.isscalar(idx)
    ids = np.ascontiguousarray(np.atleast_1d(np.asarray(idx, dtype=np.uint64)))
    if is_int:
        out = np.empty(ids.shape[0], dtype=np.int64)
        lib.orc_eval_many_i64(_ptr(Qm, ctypes.c_int64), n, _ptr(ids, ctypes.c_uint64),
                              ids.shape[0], _ptr(out, ctypes.c_int64))
    else:
        out = np.empty(ids.shape[0], dtype=np.float64)
        lib.orc_eval_many_f64(_ptr(Qm, ctypes.c_double), n, _ptr(ids, ctypes.c_uint64),
                              ids.shape[0], _ptr(out, ctypes.c_double))
    return out[0].item() if scalar else out


def brute_min(Q, lo: int = 0, hi: int | None = None, threads: int = 0):
    """(min value, argmin idx) over idx in [lo, hi), natural order, ties -> lowest idx."""
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    n = Qm.shape[0]
    if hi is None:
        hi = 1 << n
    am = ctypes.c_uint64()
    if is_int:
        v = ctypes.c_int64()
        rc = lib.orc_min_i64(_ptr(Qm, ctypes.c_int64), n, lo, hi, threads,
                             ctypes.byref(v), ctypes.byref(am))
    else:
        v = ctypes.c_double()
        rc = lib.orc_min_f64(_ptr(Qm, ctypes.c_double), n, lo, hi, threads,
                             ctypes.byref(v), ctypes.byref(am))
    if rc != 0:
        raise ValueError("oracle brute_min: bad arguments")
    return v.value, am.value


def brute_topk(Q, k: int, lo: int = 0, hi: int | None = None, threads: int = 0):
    """k smallest states by (value, idx); returns (values, indices) arrays."""
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    n = Qm.shape[0]
    if hi is None:
        hi = 1 << n
    ix = np.zeros(k, dtype=np.uint64)
    if is_int:
        vals = np.zeros(k, dtype=np.int64)
        cnt = lib.orc_topk_i64(_ptr(Qm, ctypes.c_int64), n, lo, hi, k, threads,
                               _ptr(vals, ctypes.c_int64), _ptr(ix, ctypes.c_uint64))
    else:
        vals = np.zeros(k, dtype=np.float64)
        cnt = lib.orc_topk_f64(_ptr(Qm, ctypes.c_double), n, lo, hi, k, threads,
                               _ptr(vals, ctypes.c_double), _ptr(ix, ctypes.c_uint64))
    if cnt < 0:
        raise ValueError("oracle brute_topk: bad arguments")
    return vals[:cnt], ix[:cnt]


_BLOCKED_ERR = {-1: "bad arguments (range, k, n > 62, non-finite or oversized Q)",
                -2: "out of memory",
                -3: "more than 2^24 near-tied candidate states in one thread"}


def blocked_topk(Q, k: int, lo: int = 0, hi: int | None = None, threads: int = 0,
                 return_candidates: bool = False):
    """The k smallest states by (value, idx) -- brute_topk's answer -- computed by
    the blocked natural-order walk (qubo_oracle_blocked.c), for n up to 62.

    Float Q: the blocked FP64 values only select candidates (every state within
    the rigorous rounding bound of the running k-th best); the returned values
    are the canonical FP64 values of those candidates.  Integer Q: exact int64.
    With ``return_candidates`` also returns the number of states re-evaluated.
    """
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    n = Qm.shape[0]
    if hi is None:
        hi = 1 << n
    ix = np.zeros(k, dtype=np.uint64)
    ncand = ctypes.c_uint64(0)
    if is_int:
        vals = np.zeros(k, dtype=np.int64)
        cnt = lib.orc_topk_blocked_i64(_ptr(Qm, ctypes.c_int64), n, lo, hi, k, threads,
                                       _ptr(vals, ctypes.c_int64), _ptr(ix, ctypes.c_uint64))
    else:
        vals = np.zeros(k, dtype=np.float64)
        cnt = lib.orc_topk_blocked_f64(_ptr(Qm, ctypes.c_double), n, lo, hi, k, threads,
                                       _ptr(vals, ctypes.c_double), _ptr(ix, ctypes.c_uint64),
                                       ctypes.byref(ncand))
    if cnt < 0:
        raise ValueError("oracle blocked_topk: " + _BLOCKED_ERR.get(cnt, str(cnt)))
    if return_candidates:
        return vals[:cnt], ix[:cnt], int(ncand.value)
    return vals[:cnt], ix[:cnt]


def blocked_min(Q, lo: int = 0, hi: int | None = None, threads: int = 0):
    """(min value, lowest argmin idx) over [lo, hi) -- brute_min's answer -- by the
    blocked natural-order walk."""
    vals, ix = blocked_topk(Q, 1, lo, hi, threads)
    v = vals[0].item()
    return v, int(ix[0])


def segment_minima(Q, seg: int, nseg: int, lo: int = 0, threads: int = 0):
    """Minimum and lowest argmin of each segment [lo + s*seg, lo + (s+1)*seg),
    s < nseg, by the blocked walk (one segment per thread at a time).

    Returns (values[nseg], indices[nseg]); values are int64 for integer Q and
    canonical FP64 for float Q.
    """
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    n = Qm.shape[0]
    ix = np.zeros(nseg, dtype=np.uint64)
    if is_int:
        vals = np.zeros(nseg, dtype=np.int64)
        rc = lib.orc_segmin_blocked_i64(_ptr(Qm, ctypes.c_int64), n, lo, seg, nseg, threads,
                                        _ptr(vals, ctypes.c_int64), _ptr(ix, ctypes.c_uint64))
    else:
        vals = np.zeros(nseg, dtype=np.float64)
        rc = lib.orc_segmin_blocked_f64(_ptr(Qm, ctypes.c_double), n, lo, seg, nseg, threads,
                                        _ptr(vals, ctypes.c_double), _ptr(ix, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle segment_minima: " + _BLOCKED_ERR.get(rc, str(rc)))
    return vals, ix


def logz(Q, betas, moment: bool = True, threads: int = 0):
    """log Z(beta) = log sum_x exp(-beta f(x)) and E_beta[x x^T], FP64.

    Returns (logz[nbeta], E[nbeta, n, n] or None, min value, argmin idx).
    """
    lib = _load()
    Qm, is_int = _as_matrix(Q)
    Qd = Qm.astype(np.float64)
    n = Qd.shape[0]
    b = np.ascontiguousarray(np.atleast_1d(np.asarray(betas, dtype=np.float64)))
    lz = np.zeros(b.shape[0], dtype=np.float64)
    E = np.zeros((b.shape[0], n, n), dtype=np.float64) if moment else None
    vmin = ctypes.c_double()
    am = ctypes.c_uint64()
    rc = lib.orc_logz_f64(_ptr(Qd, ctypes.c_double), n, _ptr(b, ctypes.c_double), b.shape[0],
                          threads, _ptr(lz, ctypes.c_double),
                          _ptr(E, ctypes.c_double) if moment else None,
                          ctypes.byref(vmin), ctypes.byref(am))
    if rc != 0:
        raise ValueError("oracle logz: bad arguments")
    return lz, E, vmin.value, am.value


def ising_from_qubo(Q):
    """QUBO -> Ising by x = (1 + s) / 2 (the equivalence the introduction cites).

    With W_ij = Q_ij + Q_ji for i < j:
        J_ij = W_ij / 4 (i < j, zero elsewhere)
        h_i  = Q_ii / 2 + sum_{j != i} W_{min(i,j), max(i,j)} / 4
        c    = sum_i Q_ii / 2 + sum_{i<j} W_ij / 4
    so that x^T Q x = c + h.s + sum_{i<j} J_ij s_i s_j for every x.
    """
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    W = np.triu(Qd + Qd.T, 1)
    J = W / 4.0
    d = np.diag(Qd)
    h = d / 2.0 + (W.sum(axis=0) + W.sum(axis=1)) / 4.0
    c = d.sum() / 2.0 + W.sum() / 4.0
    return J, h, c


def ising_energy(J, h, c, s):
    s = np.asarray(s, dtype=np.float64)
    return c + h @ s + s @ J @ s
