"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

None of these re-types the oracle's canonical-order sum.  Each pin comes from
somewhere else: a table evaluated by hand from Eq. 1, the f(0) = 0 fact of
Section 2.1, closed forms, the QUBO->Ising change of variables, the library
matrix product x @ Q @ x (the naive method of Section 3), and
scipy's logsumexp for the partition function.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy.special import logsumexp, expit

import oracle
from conftest import GOLDEN
from paper_2310_19373_gb300 import inputs


def _bits(n):
    """All x in natural order as an (2^n, n) 0/1 matrix, x_i = bit i of idx."""
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- hand-worked


@pytest.mark.parametrize("name", ["hand_n2.json", "hand_n3.json"])
def test_hand_worked_tables(name):
    g = _load(name)
    Q = np.array(g["Q"], dtype=np.int64)
    n = Q.shape[0]
    got = [oracle.evaluate(Q, i) for i in range(1 << n)]
    assert got == g["f_by_idx"]
    Qf = Q.astype(np.float64)
    assert [oracle.evaluate(Qf, i) for i in range(1 << n)] == [float(v) for v in g["f_by_idx"]]
    assert oracle.brute_min(Q) == (g["min"], g["argmin"])
    assert oracle.brute_min(Qf) == (float(g["min"]), g["argmin"])
    if "top3" in g:
        vals, ix = oracle.brute_topk(Q, 3)
        assert [[int(v), int(i)] for v, i in zip(vals, ix)] == g["top3"]


def test_tie_rule_differs_from_gray_first():
    """The lowest natural index wins, not the first state met in Gray order."""
    g = _load("hand_n2.json")
    v, am = oracle.brute_min(np.array(g["Q"]))
    assert am == g["argmin"] and am != g["gray_first_argmin"]


# ---------------------------------------------------------------- invariants


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_zero_vector_and_unit_vectors(seed):
    """f(0) = 0 (Section 2.1); f(e_i) = Q_ii and f(e_i+e_j) = Q_ii+Q_jj+Q_ij+Q_ji (Eq. 1)."""
    rng = np.random.default_rng(seed)
    n = 9
    for Q in (rng.normal(size=(n, n)), rng.integers(-9, 10, size=(n, n))):
        assert oracle.evaluate(Q, 0) == 0
        for i in range(n):
            assert oracle.evaluate(Q, 1 << i) == Q[i, i]
            for j in range(i + 1, n):
                want = Q[i, i] + Q[j, j] + Q[i, j] + Q[j, i]
                got = oracle.evaluate(Q, (1 << i) | (1 << j))
                assert abs(got - want) <= 1e-12 * (1 + abs(want))


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_matches_numpy_quadratic_form_int(n):
    """Exact agreement with the library product x @ Q @ x for every x (integer Q)."""
    rng = np.random.default_rng(100 + n)
    Q = rng.integers(-50, 51, size=(n, n))
    X = _bits(n)
    want = np.einsum("si,ij,sj->s", X, Q, X)
    got = oracle.evaluate(Q, np.arange(1 << n, dtype=np.uint64))
    assert np.array_equal(got, want)
    order = np.lexsort((np.arange(1 << n), want))
    assert oracle.brute_min(Q) == (int(want[order[0]]), int(order[0]))


@pytest.mark.parametrize("n", [3, 8, 11])
def test_matches_numpy_quadratic_form_float(n):
    rng = np.random.default_rng(200 + n)
    Q = np.triu(rng.uniform(-1, 1, size=(n, n)))
    X = _bits(n).astype(np.float64)
    want = np.einsum("si,ij,sj->s", X, Q, X)
    got = oracle.evaluate(Q, np.arange(1 << n, dtype=np.uint64))
    V = np.abs(Q).sum()
    assert np.max(np.abs(got - want)) <= 1e-13 * V
    v, am = oracle.brute_min(Q)
    assert am == int(np.argmin(want))
    assert abs(v - want.min()) <= 1e-13 * V


def test_lower_part_is_folded():
    """x^T L x = x^T L^T x for any L, so moving mass between Q_ij and Q_ji keeps f."""
    rng = np.random.default_rng(7)
    n = 8
    Q = np.triu(rng.integers(-20, 21, size=(n, n)))
    L = np.tril(rng.integers(-20, 21, size=(n, n)), -1)
    Q2 = Q + L - L.T
    ids = np.arange(1 << n, dtype=np.uint64)
    assert np.array_equal(oracle.evaluate(Q, ids), oracle.evaluate(Q2, ids))
    # but a transposed-only lower part (no compensation) changes f
    assert not np.array_equal(oracle.evaluate(Q, ids), oracle.evaluate(Q + L, ids))


def test_positive_scaling_keeps_argmin():
    rng = np.random.default_rng(3)
    Q = np.triu(rng.integers(-30, 31, size=(10, 10)))
    v, am = oracle.brute_min(Q)
    v3, am3 = oracle.brute_min(3 * Q)
    assert am3 == am and v3 == 3 * v


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("seed", [0, 1])
def test_diagonal_closed_form(seed):
    """Diagonal Q: min = sum_i min(0, Q_ii); x_i = 1 iff Q_ii < 0 (Q_ii = 0 -> 0, lowest index)."""
    rng = np.random.default_rng(seed)
    n = 14
    d = rng.integers(-5, 6, size=n)
    d[3] = 0
    Q = np.diag(d)
    v, am = oracle.brute_min(Q)
    assert v == np.minimum(d, 0).sum()
    assert am == sum(1 << i for i in range(n) if d[i] < 0)
    dfl = rng.uniform(-1, 1, size=n)
    Qf = np.diag(dfl)
    v, am = oracle.brute_min(Qf)
    assert am == sum(1 << i for i in range(n) if dfl[i] < 0)
    assert abs(v - np.minimum(dfl, 0).sum()) <= 1e-14 * n


def test_all_zero_matrix_ties_to_index_zero():
    for Q in (np.zeros((12, 12)), np.zeros((12, 12), dtype=np.int64)):
        assert oracle.brute_min(Q) == (0, 0)
        vals, ix = oracle.brute_topk(Q, 5)
        assert list(ix) == [0, 1, 2, 3, 4]


# ---------------------------------------------------------------- Ising


@pytest.mark.parametrize("seed", [0, 1])
def test_qubo_to_ising_energy(seed):
    """x^T Q x equals the Ising energy of s = 2x - 1 for every state; minima coincide."""
    rng = np.random.default_rng(seed)
    n = 7
    for Q in (np.triu(rng.normal(size=(n, n))), rng.integers(-9, 10, size=(n, n))):
        J, h, c = oracle.ising_from_qubo(Q)
        f = oracle.evaluate(Q, np.arange(1 << n, dtype=np.uint64))
        S = 2 * _bits(n) - 1
        E = np.array([oracle.ising_energy(J, h, c, s) for s in S])
        assert np.max(np.abs(E - f)) <= 1e-12 * (1 + np.abs(Q).sum())
        v, am = oracle.brute_min(Q)
        assert int(np.argmin(E)) == am or abs(E[am] - E.min()) <= 1e-12


# ---------------------------------------------------------------- chunking / ranges / top-k


def test_thread_count_does_not_change_result():
    Q = inputs.uniform_int(16, seed=5, lo=-3, hi=3)  # small range -> many exact ties
    ref = oracle.brute_min(Q, threads=1)
    for t in (2, 3, 7, 16):
        assert oracle.brute_min(Q, threads=t) == ref
    vals1, ix1 = oracle.brute_topk(Q, 20, threads=1)
    vals5, ix5 = oracle.brute_topk(Q, 20, threads=5)
    assert np.array_equal(vals1, vals5) and np.array_equal(ix1, ix5)


def test_ranges_and_topk_against_numpy():
    n = 10
    rng = np.random.default_rng(11)
    Q = rng.integers(-4, 5, size=(n, n))
    X = _bits(n)
    f = np.einsum("si,ij,sj->s", X, Q, X)
    order = np.lexsort((np.arange(1 << n), f))
    vals, ix = oracle.brute_topk(Q, 37)
    assert np.array_equal(ix, order[:37]) and np.array_equal(vals, f[order[:37]])
    for lo, hi in [(0, 1), (5, 6), (100, 700), (1000, 1024)]:
        sub = f[lo:hi]
        j = int(np.argmin(sub))
        assert oracle.brute_min(Q, lo, hi) == (int(sub[j]), lo + j)
    vals, ix = oracle.brute_topk(Q, 8, 3, 6)  # fewer states than k
    assert list(ix) == sorted(range(3, 6), key=lambda i: (f[i], i))


# ---------------------------------------------------------------- log Z


def test_logz_matches_scipy_logsumexp():
    n = 9
    rng = np.random.default_rng(4)
    Q = np.triu(rng.normal(0, 1 / np.sqrt(n), size=(n, n)))
    X = _bits(n).astype(np.float64)
    f = np.einsum("si,ij,sj->s", X, Q, X)
    betas = [0.1, 1.0, 10.0]
    lz, E, vmin, am = oracle.logz(Q, betas)
    for b, beta in enumerate(betas):
        assert abs(lz[b] - logsumexp(-beta * f)) <= 1e-13 * (1 + abs(lz[b]))
        w = np.exp(-beta * f - logsumexp(-beta * f))
        Ew = np.einsum("s,si,sj->ij", w, X, X)
        assert np.max(np.abs(E[b] - Ew)) <= 1e-13
    assert am == int(np.argmin(f))


def test_logz_diagonal_closed_form():
    """Diagonal Q: log Z = sum log(1 + e^{-beta Q_ii}), E[x_i] = sigmoid(-beta Q_ii), independent."""
    rng = np.random.default_rng(8)
    d = rng.uniform(-1, 1, size=10)
    Q = np.diag(d)
    betas = [0.1, 1.0, 10.0]
    lz, E, _, _ = oracle.logz(Q, betas)
    for b, beta in enumerate(betas):
        assert abs(lz[b] - np.sum(np.log1p(np.exp(-beta * d)))) <= 1e-12
        p = expit(-beta * d)
        want = np.outer(p, p)
        want[np.diag_indices(10)] = p
        assert np.max(np.abs(E[b] - want)) <= 1e-12


def test_logz_small_beta_limit():
    """beta -> 0: log Z -> n log 2 - beta * mean f, E[x_i x_j] -> 1/4 (i != j), 1/2 (i = j)."""
    n = 8
    rng = np.random.default_rng(9)
    Q = np.triu(rng.normal(size=(n, n)))
    mean_f = np.trace(Q) / 2 + np.triu(Q, 1).sum() / 4
    beta = 1e-6
    lz, E, _, _ = oracle.logz(Q, [beta])
    assert abs(lz[0] - (n * math.log(2) - beta * mean_f)) <= 1e-10
    want = np.full((n, n), 0.25)
    want[np.diag_indices(n)] = 0.5
    assert np.max(np.abs(E[0] - want)) <= 1e-5


# ---------------------------------------------------------------- planted mistakes


def _pins_hold(evaluate):
    """Run a few of the pins above against an arbitrary evaluator."""
    g3 = _load("hand_n3.json")
    if [evaluate(np.array(g3["Q"]), i) for i in range(8)] != g3["f_by_idx"]:
        return False
    rng = np.random.default_rng(0)
    Q = rng.integers(-9, 10, size=(6, 6))
    X = _bits(6)
    want = np.einsum("si,ij,sj->s", X, Q, X)
    return all(evaluate(Q, i) == want[i] for i in range(64))


def test_planted_mistakes_are_caught():
    """A dropped lower term, a swapped index or a wrong sign each break a pin."""

    def good(Q, idx):
        return oracle.evaluate(Q, idx)

    def dropped_lower(Q, idx):
        return oracle.evaluate(np.triu(Q), idx)

    def swapped(Q, idx):
        n = Q.shape[0]
        x = [(idx >> i) & 1 for i in range(n)]
        return sum(Q[i, j] * x[i] * x[(j + 1) % n] for i in range(n) for j in range(n))

    def wrong_sign(Q, idx):
        return oracle.evaluate(Q - 2 * np.diag(np.diag(Q)), idx)

    assert _pins_hold(good)
    for bad in (dropped_lower, swapped, wrong_sign):
        assert not _pins_hold(bad)


def test_logz_moment_matches_central_differences():
    """d log Z / d Q_ij = -beta E[x_i x_j]: the moment sums against differences of log Z (h = 1e-3)."""
    n = 6
    rng = np.random.default_rng(12)
    Q = np.triu(rng.normal(0, 1 / np.sqrt(n), size=(n, n)))
    h = 1e-3
    for beta in (0.1, 1.0):
        _, E, _, _ = oracle.logz(Q, [beta])
        for i, j in [(0, 0), (1, 4), (2, 5), (5, 5), (3, 1)]:
            Qp, Qm = Q.copy(), Q.copy()
            Qp[i, j] += h
            Qm[i, j] -= h
            fd = (oracle.logz(Qp, [beta], moment=False)[0][0] -
                  oracle.logz(Qm, [beta], moment=False)[0][0]) / (2 * h)
            assert abs(fd - (-beta * E[0][i, j])) <= 1e-5 * max(1e-3, abs(beta * E[0][i, j]))


# ---------------------------------------------------------------- blocked natural-order walk


def _literal_vs_blocked(Q, k, lo, hi, threads):
    a = oracle.brute_topk(Q, k, lo, hi)
    b = oracle.blocked_topk(Q, k, lo, hi, threads=threads)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (k, lo, hi, a, b)


@pytest.mark.parametrize("seed", range(6))
def test_blocked_walk_equals_literal_oracle(seed):
    """The blocked walk (the large-n oracle) returns the literal loop's top-k bit
    for bit: float Q in canonical FP64, integer Q exactly, with many exact ties
    (small integer ranges, integer-valued floats), on ragged index ranges and
    for thread counts that split blocks unevenly."""
    rng = np.random.default_rng(5000 + seed)
    for trial in range(12):
        n = int(rng.integers(1, 21))
        kind = trial % 4
        if kind == 0:
            Q = rng.integers(-3, 4, size=(n, n))
        elif kind == 1:
            Q = np.triu(rng.normal(size=(n, n)))
        elif kind == 2:
            Q = rng.integers(-1, 2, size=(n, n)).astype(np.float64)  # exact float ties
        else:
            Q = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
        N = 1 << n
        lo = int(rng.integers(0, N))
        hi = int(rng.integers(lo + 1, N + 1))
        if trial % 3 == 0:
            lo, hi = 0, N
        _literal_vs_blocked(Q, int(rng.integers(1, 40)), lo, hi, int(rng.integers(1, 9)))


def test_blocked_walk_hand_tables_and_closed_forms():
    """The hand-worked n = 2, 3 tables, the diagonal closed form and the all-zero
    matrix (every state ties at 0, lowest indices first) through the blocked walk."""
    for name in ("hand_n2.json", "hand_n3.json"):
        g = _load(name)
        for Q in (np.array(g["Q"], dtype=np.int64), np.array(g["Q"], dtype=np.float64)):
            v, am = oracle.blocked_min(Q)
            assert (v, am) == (g["min"], g["argmin"])
    d = np.random.default_rng(3).uniform(-1, 1, size=22)
    v, am = oracle.blocked_min(np.diag(d))
    assert am == sum(1 << i for i in range(22) if d[i] < 0)
    assert abs(v - np.minimum(d, 0).sum()) <= 1e-14 * 22
    for Z in (np.zeros((23, 23)), np.zeros((23, 23), dtype=np.int32)):
        vals, ix = oracle.blocked_topk(Z, 4)
        assert list(ix) == [0, 1, 2, 3] and list(vals) == [0, 0, 0, 0]


@pytest.mark.parametrize("n", [22, 24])
def test_blocked_walk_at_larger_n(n):
    """Past the 2^12-state block: several high parts per thread, top-8, against the
    literal loop (float and integer with ties)."""
    rng = np.random.default_rng(6000 + n)
    for Q in (np.triu(rng.normal(size=(n, n))).astype(np.float32),
              rng.integers(-2, 3, size=(n, n)).astype(np.int16)):
        _literal_vs_blocked(Q, 8, 0, 1 << n, 0)


def test_segment_minima_equal_range_minima():
    """Per-segment minima (the per-prefix minima of a walk with the top bits as
    the prefix) equal brute_min over each segment."""
    rng = np.random.default_rng(61)
    for Q in (rng.integers(-50, 51, size=(17, 17)), np.triu(rng.normal(size=(17, 17)))):
        for seg, nseg, lo in ((1 << 13, 16, 0), (1 << 9, 40, 3 << 9), (1, 20, 777)):
            v, ix = oracle.segment_minima(Q, seg, nseg, lo)
            for s in range(nseg):
                assert (v[s], ix[s]) == oracle.brute_min(Q, lo + s * seg, lo + (s + 1) * seg)


def test_blocked_walk_catches_planted_mistakes():
    """A dropped lower part or a wrong sign in Q changes the blocked answer on an
    instance whose literal answer is known, so the comparison above has teeth."""
    rng = np.random.default_rng(62)
    n = 15
    Q = rng.integers(-9, 10, size=(n, n))
    ref = oracle.brute_topk(Q, 5)
    for bad in (np.triu(Q), Q - 2 * np.diag(np.diag(Q))):
        got = oracle.blocked_topk(bad, 5)
        assert not (np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]))
