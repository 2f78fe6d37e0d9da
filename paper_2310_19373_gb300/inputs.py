"""Seeded synthetic QUBO generators.

These build the input matrices that both the GPU library and the CPU oracle
are run on.  They only draw random numbers and lay them out; none of the
method's arithmetic lives here, and nothing here imports the CUDA binding.

The paper's experiments use "random QUBO instances" with no stated
distribution (Section 3, Fig. 2), so the workloads are the synthetic
distributions below, all upper triangular (Eq. 1 takes Q upper triangular),
drawn with numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np


def upper(M: np.ndarray) -> np.ndarray:
    return np.triu(M)


def uniform_f64(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n x n, entries i.i.d. uniform[lo, hi] on i <= j (diagonal included), 0 below."""
    rng = np.random.default_rng(seed)
    return upper(rng.uniform(lo, hi, size=(n, n))).astype(np.float64)


def uniform_int(n: int, seed: int = 0, lo: int = -100, hi: int = 100,
                dtype=np.int32, sparsity: float = 0.0, mask_seed: int = 1) -> np.ndarray:
    """n x n integer entries i.i.d. uniform in [lo, hi] on i <= j.

    With ``sparsity`` p > 0 every off-diagonal entry is zeroed with
    probability p, using its own stream ``mask_seed``.
    """
    rng = np.random.default_rng(seed)
    Q = upper(rng.integers(lo, hi + 1, size=(n, n))).astype(dtype)
    if sparsity > 0.0:
        mrng = np.random.default_rng(mask_seed)
        drop = mrng.random(size=(n, n)) < sparsity
        np.fill_diagonal(drop, False)
        Q[drop] = 0
    return Q


def gaussian_f32(n: int, seed: int = 0, off_mean: float = 0.0, off_std: float = 1.0,
                 diag_mean: float = -0.5, diag_std: float = 1.0) -> np.ndarray:
    """Off-diagonal N(off_mean, off_std^2), diagonal N(diag_mean, diag_std^2), upper, FP32."""
    rng = np.random.default_rng(seed)
    M = rng.normal(off_mean, off_std, size=(n, n))
    d = rng.normal(diag_mean, diag_std, size=n)
    M[np.diag_indices(n)] = d
    return upper(M).astype(np.float32)


# ---- the five workloads -------------------------------------------------

def config_n20_f64(seed: int = 0) -> np.ndarray:
    """n=20, FP64 uniform[-1,1] upper triangular (diagonal included)."""
    return uniform_f64(20, seed)


def config_n32_int(seed: int = 0, sparse: bool = False) -> np.ndarray:
    """n=32, int32 uniform integers in [-100, 100]; optional 50% off-diagonal sparsity."""
    return uniform_int(32, seed, -100, 100, np.int32, 0.5 if sparse else 0.0, mask_seed=1)


def config_n40_f32(seed: int = 0) -> np.ndarray:
    """n=40, FP32, off-diagonal N(0,1), diagonal N(-0.5,1), upper."""
    return gaussian_f32(40, seed, 0.0, 1.0, -0.5, 1.0)


def config_batched(count: int = 4096, n_lo: int = 16, n_hi: int = 34, seed: int = 0):
    """Batch of ``count`` instances, n_i uniform in {n_lo..n_hi}.

    The first half is FP32 uniform[-1,1]; the second half holds int16 values
    uniform in {-50..50}.  One stream (``seed``), instance order fixed.
    Returns a list of numpy matrices (float32 or int16).
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for i, n in enumerate(ns):
        n = int(n)
        if i < count // 2:
            out.append(upper(rng.uniform(-1.0, 1.0, size=(n, n))).astype(np.float32))
        else:
            out.append(upper(rng.integers(-50, 51, size=(n, n))).astype(np.int16))
    return out


def config_logz(count: int = 64, n: int = 28, seed: int = 0) -> np.ndarray:
    """``count`` FP32 instances at n, entries N(0, 1/n) upper; shape (count, n, n)."""
    rng = np.random.default_rng(seed)
    Q = rng.normal(0.0, 1.0 / np.sqrt(n), size=(count, n, n))
    return np.triu(Q).astype(np.float32)


LOGZ_BETAS = (0.1, 1.0, 10.0)
