"""ctypes binding of libqubobf (include/qbf.h).

Argument marshalling only: every step of a solve runs in the CUDA library.
The low-level functions keep the C names; ``solve`` is a convenience wrapper
that takes a torch tensor (device or host) and returns a ``Solution``.
If the library has not been built this module raises on first use -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqubobf.so")

QBF_F64, QBF_F32, QBF_I32, QBF_I16 = 0, 1, 2, 3
QBF_OK, QBF_EINVAL, QBF_ENONFINITE, QBF_EDTYPE, QBF_ECUDA = 0, 1, 2, 3, 4
QBF_EOVERFLOW, QBF_ECANCELED, QBF_ENOTIMPL, QBF_ERANGE = 5, 6, 7, 8
QBF_VARIANT_AUTO, QBF_VARIANT_FIELD, QBF_VARIANT_SPLIT, QBF_VARIANT_TC = 0, 1, 2, 3
QBF_VARIANT_SPLIT_F32 = 4
QBF_VARIANT_SPLIT_MIX = 5
QBF_VARIANT_NAIVE = 6
QBF_VARIANT_SPLIT_DEFER = 7
QBF_MAX_N = 48
QBF_MAX_TOPK = 64

STATUS_NAMES = {
    0: "QBF_OK", 1: "QBF_EINVAL", 2: "QBF_ENONFINITE", 3: "QBF_EDTYPE", 4: "QBF_ECUDA",
    5: "QBF_EOVERFLOW", 6: "QBF_ECANCELED", 7: "QBF_ENOTIMPL", 8: "QBF_ERANGE",
}


class QbfOptions(ctypes.Structure):
    _fields_ = [
        ("top_k", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("prefix_bits", ctypes.c_int),
        ("fix_bits", ctypes.c_int),
        ("fix_value", ctypes.c_uint64),
        ("timing", ctypes.c_int),
        ("batch_suffix_bits", ctypes.c_int),
        ("reserved", ctypes.c_int * 6),
    ]


class QbfResult(ctypes.Structure):
    _fields_ = [
        ("min_value", ctypes.c_double),
        ("argmin", ctypes.c_uint64),
        ("top_k", ctypes.c_int),
        ("topk_value", ctypes.c_double * QBF_MAX_TOPK),
        ("topk_index", ctypes.c_uint64 * QBF_MAX_TOPK),
        ("scale_bits", ctypes.c_int),
        ("error_bound", ctypes.c_double),
        ("n_candidates", ctypes.c_uint64),
        ("prefix_bits", ctypes.c_int),
        ("suffix_bits", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("walk_launches", ctypes.c_int),
        ("walk_seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_int),
        ("reserved", ctypes.c_int * 3),
    ]


class QbfBatchInfo(ctypes.Structure):
    _fields_ = [
        ("error_bound", ctypes.c_double),
        ("n_candidates", ctypes.c_uint64),
        ("scale_bits", ctypes.c_int),
        ("suffix_bits", ctypes.c_int),
        ("prefix_bits", ctypes.c_int),
        ("walk", ctypes.c_int),
    ]


QBF_CKPT_VERSION = 1


class QbfCheckpoint(ctypes.Structure):
    _fields_ = [
        ("version", ctypes.c_uint32),
        ("n", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("top_k", ctypes.c_int32),
        ("chunk_bits", ctypes.c_int32),
        ("shard", ctypes.c_int32),
        ("nshards", ctypes.c_int32),
        ("count", ctypes.c_int32),
        ("q_hash", ctypes.c_uint64),
        ("next", ctypes.c_uint64),
        ("chunks_done", ctypes.c_uint64),
        ("done_mask", ctypes.c_uint64),
        ("n_candidates", ctypes.c_uint64),
        ("error_bound", ctypes.c_double),
        ("best_value", ctypes.c_double * QBF_MAX_TOPK),
        ("best_index", ctypes.c_uint64 * QBF_MAX_TOPK),
    ]


class QbfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_VP = ctypes.c_void_p
_SIGS = {
    "qbf_default_options": (None, [ctypes.POINTER(QbfOptions)]),
    "qbf_solve": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(QbfOptions),
                                 ctypes.POINTER(QbfResult), _VP]),
    "qbf_solve_host": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(QbfOptions), ctypes.POINTER(QbfResult), _VP]),
    "qbf_chunked_init": (ctypes.c_int, [ctypes.POINTER(QbfCheckpoint), _VP, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _VP]),
    "qbf_chunked_step": (ctypes.c_int, [ctypes.POINTER(QbfCheckpoint), _VP,
                                        ctypes.POINTER(QbfOptions), ctypes.c_uint64, _VP]),
    "qbf_chunked_merge": (ctypes.c_int, [ctypes.POINTER(QbfCheckpoint),
                                         ctypes.POINTER(QbfCheckpoint)]),
    "qbf_chunked_result": (ctypes.c_int, [ctypes.POINTER(QbfCheckpoint),
                                          ctypes.POINTER(QbfResult)]),
    "qubo_bf_solve": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int)]),
    "qbf_solve_ising": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(QbfOptions), ctypes.POINTER(QbfResult), _VP]),
    "qbf_solve_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                         ctypes.POINTER(QbfOptions), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint64), _VP]),
    "qbf_solve_batched_info": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                              ctypes.POINTER(QbfOptions),
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(QbfBatchInfo), _VP]),
    "qbf_solve_batched_item_minima": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                                     ctypes.POINTER(ctypes.c_int),
                                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                     ctypes.POINTER(QbfOptions), ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.c_uint64,
                                                     ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(QbfBatchInfo), _VP]),
    "qbf_cancel": (ctypes.c_int, []),
    "qbf_tune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_char_p]),
    "qbf_tuned_params": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "qbf_tune_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double), _VP]),
    "qbf_logz": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_uint64), _VP]),
    "qbf_logz_backward": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int, _VP, _VP,
                                         _VP, _VP]),
    "qbf_danskin": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int,
                                   _VP, _VP, _VP]),
    "qbf_solve_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(QbfOptions), ctypes.POINTER(QbfResult),
                                         _VP]),
    "qbf_walk_trace": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                      ctypes.POINTER(ctypes.c_int), _VP]),
    "qbf_prefix_minima": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int), _VP]),
    "qbf_prefix_minima_fixed": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _VP,
                                               ctypes.POINTER(ctypes.c_int), _VP]),
    "qbf_tc_selftest": (ctypes.c_int, [_VP, _VP, _VP]),
    "qbf_alu_microbench": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), _VP]),
    "qbf_last_error_string": (ctypes.c_char_p, []),
    "qbf_release": (ctypes.c_int, []),
    "qbf_version": (ctypes.c_int, []),
}


def lib():
    """Load libqubobf.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != QBF_OK:
        raise QbfError(rc, lib().qbf_last_error_string().decode(errors="replace"))


# ---- same names as the C ABI ---------------------------------------------


def qbf_default_options() -> QbfOptions:
    o = QbfOptions()
    lib().qbf_default_options(ctypes.byref(o))
    return o


def qbf_solve(Q_dev: int, n: int, dtype: int, opt: QbfOptions | None, stream: int | None = None):
    out = QbfResult()
    rc = lib().qbf_solve(_VP(Q_dev), n, dtype, ctypes.byref(opt) if opt is not None else None,
                         ctypes.byref(out), _VP(stream or 0))
    _check(rc)
    return out


def qbf_solve_host(Q_host: int, n: int, dtype: int, opt: QbfOptions | None,
                   stream: int | None = None):
    out = QbfResult()
    rc = lib().qbf_solve_host(_VP(Q_host), n, dtype,
                              ctypes.byref(opt) if opt is not None else None,
                              ctypes.byref(out), _VP(stream or 0))
    _check(rc)
    return out


def qbf_solve_ising(J_dev: int, h_dev: int, n: int, dtype: int, opt: QbfOptions | None,
                    stream: int | None = None):
    out = QbfResult()
    rc = lib().qbf_solve_ising(_VP(J_dev), _VP(h_dev), n, dtype,
                               ctypes.byref(opt) if opt is not None else None,
                               ctypes.byref(out), _VP(stream or 0))
    _check(rc)
    return out


def qubo_bf_solve(Q, top_k: int = 0):
    """The one-call form for a host matrix (numpy array or CPU tensor): returns
    (min_value, argmin, [(value, index), ...] of the top_k best states)."""
    import numpy as np

    a = np.ascontiguousarray(Q.numpy() if hasattr(Q, "numpy") else Q)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise QbfError(QBF_EINVAL, "Q must be a square matrix")
    codes = {np.dtype(np.float64): QBF_F64, np.dtype(np.float32): QBF_F32,
             np.dtype(np.int32): QBF_I32, np.dtype(np.int16): QBF_I16}
    if a.dtype not in codes:
        raise QbfError(QBF_EDTYPE, f"unsupported dtype {a.dtype}")
    vmin, am, cnt = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_int()
    tv = (ctypes.c_double * max(top_k, 1))()
    ti = (ctypes.c_uint64 * max(top_k, 1))()
    _check(lib().qubo_bf_solve(_VP(a.ctypes.data), a.shape[0], codes[a.dtype], ctypes.byref(vmin),
                               ctypes.byref(am), top_k, tv, ti, ctypes.byref(cnt)))
    return vmin.value, int(am.value), [(tv[i], int(ti[i])) for i in range(cnt.value)]


def qbf_chunked_init(ck: QbfCheckpoint, Q_dev: int, n: int, dtype: int, top_k: int,
                     chunk_bits: int, shard: int = 0, nshards: int = 1, stream: int | None = None):
    _check(lib().qbf_chunked_init(ctypes.byref(ck), _VP(Q_dev), n, dtype, top_k, chunk_bits,
                                  shard, nshards, _VP(stream or 0)))


def qbf_chunked_step(ck: QbfCheckpoint, Q_dev: int, opt: QbfOptions | None, max_chunks: int,
                     stream: int | None = None):
    _check(lib().qbf_chunked_step(ctypes.byref(ck), _VP(Q_dev),
                                  ctypes.byref(opt) if opt is not None else None,
                                  max_chunks, _VP(stream or 0)))


def qbf_chunked_merge(into: QbfCheckpoint, other: QbfCheckpoint):
    _check(lib().qbf_chunked_merge(ctypes.byref(into), ctypes.byref(other)))


def qbf_chunked_result(ck: QbfCheckpoint) -> QbfResult:
    out = QbfResult()
    _check(lib().qbf_chunked_result(ctypes.byref(ck), ctypes.byref(out)))
    return out


def _batch_arrays(Q_ptrs, ns, dtypes):
    count = len(Q_ptrs)
    P = (ctypes.c_void_p * count)(*[ctypes.c_void_p(int(q)) for q in Q_ptrs])
    N = (ctypes.c_int * count)(*[int(v) for v in ns])
    D = (ctypes.c_int * count)(*[int(v) for v in dtypes])
    return count, P, N, D


def qbf_solve_batched(Q_ptrs, ns, dtypes, opt: QbfOptions | None, stream: int | None = None):
    """Q_ptrs: device pointers; returns (min_values, argmins) as lists."""
    count, P, N, D = _batch_arrays(Q_ptrs, ns, dtypes)
    vmin = (ctypes.c_double * count)()
    am = (ctypes.c_uint64 * count)()
    rc = lib().qbf_solve_batched(P, N, D, count, ctypes.byref(opt) if opt is not None else None,
                                 vmin, am, _VP(stream or 0))
    _check(rc)
    return list(vmin), [int(v) for v in am]


def qbf_solve_batched_info(Q_ptrs, ns, dtypes, opt: QbfOptions | None,
                           stream: int | None = None):
    """As qbf_solve_batched, plus one QbfBatchInfo per instance."""
    count, P, N, D = _batch_arrays(Q_ptrs, ns, dtypes)
    vmin = (ctypes.c_double * count)()
    am = (ctypes.c_uint64 * count)()
    info = (QbfBatchInfo * count)()
    rc = lib().qbf_solve_batched_info(P, N, D, count,
                                      ctypes.byref(opt) if opt is not None else None, vmin, am,
                                      info, _VP(stream or 0))
    _check(rc)
    return list(vmin), [int(v) for v in am], list(info)


def qbf_solve_batched_item_minima(Q_ptrs, ns, dtypes, opt: QbfOptions | None, inst: int,
                                  max_items: int, stream: int | None = None):
    """Per-item minima of instance `inst` (items of 32 prefixes) and the batch's
    QbfBatchInfo list; see include/qbf.h."""
    count, P, N, D = _batch_arrays(Q_ptrs, ns, dtypes)
    out = (ctypes.c_int32 * max(1, max_items))()
    nit = ctypes.c_uint64()
    info = (QbfBatchInfo * count)()
    rc = lib().qbf_solve_batched_item_minima(P, N, D, count,
                                             ctypes.byref(opt) if opt is not None else None,
                                             inst, out, max_items, ctypes.byref(nit), info,
                                             _VP(stream or 0))
    _check(rc)
    return list(out[:min(max_items, nit.value)]), nit.value, list(info)


def batched_item_minima(Qs, inst: int, max_items: int, batch_suffix_bits: int = 0,
                        stream=None, variant: int = QBF_VARIANT_AUTO):
    """Per-item minima of instance `inst` of a batched solve of square CUDA
    tensors: (item minima, item count, per-instance QbfBatchInfo)."""
    import torch

    Qs = [q.contiguous() for q in Qs]
    opt = qbf_default_options()
    opt.batch_suffix_bits = batch_suffix_bits
    opt.variant = variant
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    return qbf_solve_batched_item_minima([q.data_ptr() for q in Qs], [q.shape[0] for q in Qs],
                                         [dtype_code(q) for q in Qs], opt, inst, max_items, s)


def qbf_cancel() -> None:
    """Stop the running solve from any thread (it returns QBF_ECANCELED)."""
    _check(lib().qbf_cancel())


def qbf_tune(n_min: int, n_max: int, dtype: int, cache_path: str | None = None) -> None:
    """Tune the batched solver per n (suffix width, CTAs per SM); see include/qbf.h."""
    _check(lib().qbf_tune(n_min, n_max, dtype,
                          cache_path.encode() if cache_path is not None else None))


def qbf_tuned_params(n: int, dtype: int):
    """(suffix bits, CTAs per SM) the batched solver uses for n and dtype; 0 = default."""
    ns, ctas = ctypes.c_int(), ctypes.c_int()
    _check(lib().qbf_tuned_params(n, dtype, ctypes.byref(ns), ctypes.byref(ctas)))
    return ns.value, ctas.value


def qbf_tune_batched(Q_ptrs, ns, dtypes, lo_bits: int = 6, hi_bits: int = 16,
                     stream: int | None = None):
    count, P, N, D = _batch_arrays(Q_ptrs, ns, dtypes)
    best = ctypes.c_int()
    sec = ctypes.c_double()
    rc = lib().qbf_tune_batched(P, N, D, count, lo_bits, hi_bits, ctypes.byref(best),
                                ctypes.byref(sec), _VP(stream or 0))
    _check(rc)
    return best.value, sec.value


def solve_batched_info(Qs, batch_suffix_bits: int = 0, stream=None,
                       variant: int = QBF_VARIANT_AUTO):
    """Like solve_batched; returns (min_values, argmins, per-instance QbfBatchInfo)."""
    import torch

    Qs = [q.contiguous() for q in Qs]
    opt = qbf_default_options()
    opt.batch_suffix_bits = batch_suffix_bits
    opt.variant = variant
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    return qbf_solve_batched_info([q.data_ptr() for q in Qs], [q.shape[0] for q in Qs],
                                  [dtype_code(q) for q in Qs], opt, s)


def solve_batched(Qs, batch_suffix_bits: int = 0, stream=None, variant: int = QBF_VARIANT_AUTO):
    """Minimise a list of square CUDA tensors; returns (min_values, argmins)."""
    import torch

    Qs = [q.contiguous() for q in Qs]
    opt = qbf_default_options()
    opt.batch_suffix_bits = batch_suffix_bits
    opt.variant = variant
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    return qbf_solve_batched([q.data_ptr() for q in Qs], [q.shape[0] for q in Qs],
                             [dtype_code(q) for q in Qs], opt, s)


def qbf_logz(Q_dev: int, n: int, dtype: int, batch: int, betas, stream: int | None = None):
    """Returns (logz[batch][nbeta], min_values[batch], argmins[batch])."""
    nb = len(betas)
    B = (ctypes.c_double * nb)(*[float(b) for b in betas])
    lz = (ctypes.c_double * (batch * nb))()
    vm = (ctypes.c_double * batch)()
    am = (ctypes.c_uint64 * batch)()
    rc = lib().qbf_logz(_VP(Q_dev), n, dtype, batch, B, nb, lz, vm, am, _VP(stream or 0))
    _check(rc)
    return ([list(lz[b * nb:(b + 1) * nb]) for b in range(batch)], list(vm),
            [int(v) for v in am])


def qbf_logz_backward(Q_dev: int, n: int, dtype: int, batch: int, betas, upstream_dev,
                      grad_dev: int, moment_dev, stream: int | None = None) -> None:
    nb = len(betas)
    B = (ctypes.c_double * nb)(*[float(b) for b in betas])
    rc = lib().qbf_logz_backward(_VP(Q_dev), n, dtype, batch, B, nb, _VP(upstream_dev or 0),
                                 _VP(grad_dev), _VP(moment_dev or 0), _VP(stream or 0))
    _check(rc)


def qbf_danskin(argmins, n: int, batch: int, upstream_dev, grad_dev: int,
                stream: int | None = None) -> None:
    A = (ctypes.c_uint64 * batch)(*[int(a) for a in argmins])
    rc = lib().qbf_danskin(A, n, batch, _VP(upstream_dev or 0), _VP(grad_dev), _VP(stream or 0))
    _check(rc)


def qbf_solve_noalloc(Q_dev: int, n: int, dtype: int, opt: QbfOptions | None,
                      stream: int | None = None):
    """qbf_solve on the library's fixed scratch: for callers that cannot allocate GPU memory."""
    out = QbfResult()
    rc = lib().qbf_solve_noalloc(_VP(Q_dev), n, dtype,
                                 ctypes.byref(opt) if opt is not None else None,
                                 ctypes.byref(out), _VP(stream or 0))
    _check(rc)
    return out


def qbf_walk_trace(Q_dev: int, n: int, dtype: int, prefix_bits: int, idx_dev: int, val_dev: int,
                   stream: int | None = None) -> int:
    sigma = ctypes.c_int()
    rc = lib().qbf_walk_trace(_VP(Q_dev), n, dtype, prefix_bits, _VP(idx_dev), _VP(val_dev),
                              ctypes.byref(sigma), _VP(stream or 0))
    _check(rc)
    return sigma.value


def qbf_prefix_minima(Q_dev: int, n: int, dtype: int, prefix_bits: int, variant: int,
                      pmin_dev: int, stream: int | None = None) -> int:
    sigma = ctypes.c_int()
    rc = lib().qbf_prefix_minima(_VP(Q_dev), n, dtype, prefix_bits, variant, _VP(pmin_dev),
                                 ctypes.byref(sigma), _VP(stream or 0))
    _check(rc)
    return sigma.value


def qbf_prefix_minima_fixed(Q_dev: int, n: int, dtype: int, prefix_bits: int, variant: int,
                            fix_bits: int, fix_value: int, pmin_dev: int,
                            stream: int | None = None) -> int:
    sigma = ctypes.c_int()
    rc = lib().qbf_prefix_minima_fixed(_VP(Q_dev), n, dtype, prefix_bits, variant, fix_bits,
                                       fix_value, _VP(pmin_dev), ctypes.byref(sigma),
                                       _VP(stream or 0))
    _check(rc)
    return sigma.value


def qbf_tc_selftest(A_fp16_bits, B_fp16_bits):
    """A: 128x16, B: 16x128 uint16 arrays of FP16 bit patterns (numpy); returns D 128x128."""
    import numpy as np

    A = np.ascontiguousarray(A_fp16_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_fp16_bits, dtype=np.uint16)
    D = np.zeros((128, 128), dtype=np.float32)
    _check(lib().qbf_tc_selftest(A.ctypes.data, B.ctypes.data, D.ctypes.data))
    return D


def qbf_alu_microbench(op: int, stream: int | None = None):
    ops = ctypes.c_double()
    mhz = ctypes.c_double()
    sec = ctypes.c_double()
    rc = lib().qbf_alu_microbench(op, ctypes.byref(ops), ctypes.byref(mhz), ctypes.byref(sec),
                                  _VP(stream or 0))
    _check(rc)
    return ops.value, mhz.value, sec.value


def qbf_last_error_string() -> str:
    return lib().qbf_last_error_string().decode(errors="replace")


def qbf_release() -> None:
    _check(lib().qbf_release())


def qbf_version() -> int:
    return lib().qbf_version()


# ---- torch convenience ---------------------------------------------------


def dtype_code(t) -> int:
    import torch

    m = {torch.float64: QBF_F64, torch.float32: QBF_F32, torch.int32: QBF_I32,
         torch.int16: QBF_I16}
    if t.dtype not in m:
        raise QbfError(QBF_EDTYPE, f"unsupported dtype {t.dtype}")
    return m[t.dtype]


@dataclass
class Solution:
    min_value: float
    argmin: int
    topk_values: list = field(default_factory=list)
    topk_indices: list = field(default_factory=list)
    scale_bits: int = 0
    error_bound: float = 0.0
    n_candidates: int = 0
    prefix_bits: int = 0
    suffix_bits: int = 0
    variant: int = 0
    walk_launches: int = 0
    walk_seconds: float = 0.0
    kernel_launches: int = 0

    def x(self, n: int):
        """argmin as a 0/1 list, x_i = bit i of the natural index."""
        return [(self.argmin >> i) & 1 for i in range(n)]

    def spins(self, n: int):
        """argmin of an Ising solve as spins, s_i = 2 x_i - 1."""
        return [2 * b - 1 for b in self.x(n)]


def _solution(r: QbfResult) -> Solution:
    k = r.top_k
    return Solution(r.min_value, int(r.argmin), list(r.topk_value[:k]),
                    [int(v) for v in r.topk_index[:k]], r.scale_bits, r.error_bound,
                    int(r.n_candidates), r.prefix_bits, r.suffix_bits, r.variant,
                    r.walk_launches, r.walk_seconds, r.kernel_launches)


def make_options(top_k: int = 1, variant: int = QBF_VARIANT_AUTO, prefix_bits: int = -1,
                 fix_bits: int = 0, fix_value: int = 0, timing: bool = False) -> QbfOptions:
    o = qbf_default_options()
    o.timing = 1 if timing else 0
    o.top_k = top_k
    o.variant = variant
    o.prefix_bits = prefix_bits
    o.fix_bits = fix_bits
    o.fix_value = fix_value
    return o


def solve(Q, top_k: int = 1, variant: int = QBF_VARIANT_AUTO, prefix_bits: int = -1,
          fix_bits: int = 0, fix_value: int = 0, stream=None, timing: bool = False) -> Solution:
    """Minimise x^T Q x for a square torch tensor Q (CUDA or CPU memory)."""
    import torch

    if Q.dim() != 2 or Q.shape[0] != Q.shape[1]:
        raise QbfError(QBF_EINVAL, "Q must be a square matrix")
    Q = Q.contiguous()
    n = Q.shape[0]
    opt = make_options(top_k, variant, prefix_bits, fix_bits, fix_value, timing)
    if Q.is_cuda:
        s = stream if stream is not None else torch.cuda.current_stream(Q.device).cuda_stream
        with torch.cuda.device(Q.device):
            r = qbf_solve(Q.data_ptr(), n, dtype_code(Q), opt, s)
    else:
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        r = qbf_solve_host(Q.data_ptr(), n, dtype_code(Q), opt, s)
    return _solution(r)


def solve_ising(J, h, top_k: int = 1, variant: int = QBF_VARIANT_AUTO, stream=None) -> Solution:
    """Minimise E(s) = s^T J s + h^T s over s in {-1, +1}^n for CUDA tensors J
    (n x n) and h (n) of one dtype; indices have bit i = 1 iff s_i = +1
    (Solution.spins turns one into the spin vector)."""
    import torch

    if J.dim() != 2 or J.shape[0] != J.shape[1] or h.shape != (J.shape[0],):
        raise QbfError(QBF_EINVAL, "J must be n x n and h of length n")
    if J.dtype != h.dtype or not (J.is_cuda and h.is_cuda):
        raise QbfError(QBF_EINVAL, "J and h must be CUDA tensors of one dtype")
    J, h = J.contiguous(), h.contiguous()
    opt = make_options(top_k, variant, -1, 0, 0, False)
    s = stream if stream is not None else torch.cuda.current_stream(J.device).cuda_stream
    with torch.cuda.device(J.device):
        r = qbf_solve_ising(J.data_ptr(), h.data_ptr(), J.shape[0], dtype_code(J), opt, s)
    return _solution(r)


class Chunked:
    """Resumable enumeration of one QUBO in 2^chunk_bits chunks (shard `shard`
    of `nshards`).  The state is a plain qbf_checkpoint: to_bytes() after any
    step, from_bytes() to resume (in this or another process)."""

    def __init__(self, ck: QbfCheckpoint):
        self.ck = ck

    @classmethod
    def start(cls, Q, chunk_bits: int, top_k: int = 1, shard: int = 0, nshards: int = 1):
        import torch

        Q = Q.contiguous()
        ck = QbfCheckpoint()
        s = torch.cuda.current_stream(Q.device).cuda_stream
        with torch.cuda.device(Q.device):
            qbf_chunked_init(ck, Q.data_ptr(), Q.shape[0], dtype_code(Q), top_k, chunk_bits,
                             shard, nshards, s)
        return cls(ck)

    def step(self, Q, max_chunks: int, variant: int = QBF_VARIANT_AUTO) -> bool:
        """Walk up to max_chunks chunks; True once this shard is finished."""
        import torch

        Q = Q.contiguous()
        s = torch.cuda.current_stream(Q.device).cuda_stream
        with torch.cuda.device(Q.device):
            qbf_chunked_step(self.ck, Q.data_ptr(), make_options(variant=variant), max_chunks, s)
        return self.finished

    @property
    def finished(self) -> bool:
        return bool(self.ck.done_mask >> self.ck.shard & 1)

    def merge(self, other: "Chunked") -> "Chunked":
        qbf_chunked_merge(self.ck, other.ck)
        return self

    def result(self) -> Solution:
        return _solution(qbf_chunked_result(self.ck))

    def to_bytes(self) -> bytes:
        return ctypes.string_at(ctypes.addressof(self.ck), ctypes.sizeof(self.ck))

    @classmethod
    def from_bytes(cls, b: bytes) -> "Chunked":
        if len(b) != ctypes.sizeof(QbfCheckpoint):
            raise QbfError(QBF_EINVAL, "not a serialized qbf_checkpoint")
        return cls(QbfCheckpoint.from_buffer_copy(b))


def prefix_minima(Q, prefix_bits: int, variant: int = QBF_VARIANT_AUTO):
    """Per-prefix minima of the fixed-point objective from the MIN kernel, and sigma."""
    import torch

    Q = Q.contiguous()
    n = Q.shape[0]
    pm = torch.empty(1 << prefix_bits, dtype=torch.int32, device=Q.device)
    s = torch.cuda.current_stream(Q.device).cuda_stream
    sigma = qbf_prefix_minima(Q.data_ptr(), n, dtype_code(Q), prefix_bits, variant,
                              pm.data_ptr(), s)
    return pm, sigma


def prefix_minima_fixed(Q, prefix_bits: int, fix_bits: int, fix_value: int,
                        variant: int = QBF_VARIANT_AUTO):
    """Per-prefix minima over the prefixes under the top fix_bits = fix_value, and sigma."""
    import torch

    Q = Q.contiguous()
    n = Q.shape[0]
    pm = torch.empty(1 << (prefix_bits - fix_bits), dtype=torch.int32, device=Q.device)
    s = torch.cuda.current_stream(Q.device).cuda_stream
    sigma = qbf_prefix_minima_fixed(Q.data_ptr(), n, dtype_code(Q), prefix_bits, variant,
                                    fix_bits, fix_value, pm.data_ptr(), s)
    return pm, sigma


def walk_trace(Q, prefix_bits: int):
    """Every state the walk visits, as (natural index, fixed-point value, sigma) tensors."""
    import torch

    Q = Q.contiguous()
    n = Q.shape[0]
    idx = torch.empty(1 << n, dtype=torch.int64, device=Q.device)
    val = torch.empty(1 << n, dtype=torch.int64, device=Q.device)
    s = torch.cuda.current_stream(Q.device).cuda_stream
    sigma = qbf_walk_trace(Q.data_ptr(), n, dtype_code(Q), prefix_bits, idx.data_ptr(),
                           val.data_ptr(), s)
    return idx, val, sigma


# ---- differentiable wrappers ---------------------------------------------


def _autograd():
    import torch

    class LogZFn(torch.autograd.Function):
        """log Z(Q_b, beta_j) for a batch Q of shape (batch, n, n); the backward
        pass re-walks the enumeration on the GPU (qbf_logz_backward)."""

        @staticmethod
        def forward(ctx, Q, betas):
            Qc = Q.detach().contiguous()
            batch, n = Qc.shape[0], Qc.shape[1]
            s = torch.cuda.current_stream(Qc.device).cuda_stream
            lz, vmin, am = qbf_logz(Qc.data_ptr(), n, dtype_code(Qc), batch, betas, s)
            ctx.save_for_backward(Qc)
            ctx.betas = tuple(float(b) for b in betas)
            return torch.tensor(lz, dtype=torch.float64, device=Q.device)

        @staticmethod
        def backward(ctx, g):
            (Qc,) = ctx.saved_tensors
            batch, n = Qc.shape[0], Qc.shape[1]
            up = g.detach().to(torch.float64).contiguous()
            grad = torch.empty((batch, n, n), dtype=torch.float64, device=Qc.device)
            s = torch.cuda.current_stream(Qc.device).cuda_stream
            qbf_logz_backward(Qc.data_ptr(), n, dtype_code(Qc), batch, ctx.betas, up.data_ptr(),
                              grad.data_ptr(), None, s)
            return grad.to(Qc.dtype), None

    class MinFn(torch.autograd.Function):
        """min_x x^T Q_b x for a batch; backward is the Danskin subgradient x* x*^T."""

        @staticmethod
        def forward(ctx, Q):
            Qc = Q.detach().contiguous()
            vmin, am = solve_batched(list(Qc))
            ctx.argmin = am
            ctx.n = Qc.shape[1]
            ctx.dtype = Qc.dtype
            return torch.tensor(vmin, dtype=torch.float64, device=Q.device)

        @staticmethod
        def backward(ctx, g):
            batch = len(ctx.argmin)
            up = g.detach().to(torch.float64).contiguous()
            grad = torch.empty((batch, ctx.n, ctx.n), dtype=torch.float64, device=g.device)
            s = torch.cuda.current_stream(g.device).cuda_stream
            qbf_danskin(ctx.argmin, ctx.n, batch, up.data_ptr(), grad.data_ptr(), s)
            return grad.to(ctx.dtype)

    return LogZFn, MinFn


def logz(Q, betas):
    """Differentiable log Z for Q of shape (batch, n, n) on the GPU: (batch, len(betas))."""
    LogZFn, _ = _autograd()
    return LogZFn.apply(Q, tuple(betas))


def qubo_min(Q):
    """Differentiable (Danskin) minimum for Q of shape (batch, n, n): (batch,)."""
    _, MinFn = _autograd()
    return MinFn.apply(Q)
