"""GPU parity: the CUDA walk (through the C ABI) against the CPU oracle.

Integer Q must agree bit for bit; float Q is certified, so min and argmin are
those of the FP64 canonical objective and must agree exactly as well (the
oracle and the GPU rescorer use the same written summation order).
"""
import json
import os

import numpy as np
import pytest

import oracle
from conftest import GOLDEN
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def check_against_oracle(Q, top_k=1, **kw):
    sol = qb.solve(dev(Q), top_k=top_k, **kw)
    vals, ix = oracle.brute_topk(Q, top_k)
    assert sol.topk_indices == [int(i) for i in ix], (sol, vals, ix)
    assert sol.topk_values == [float(v) for v in vals]
    assert sol.min_value == float(vals[0]) and sol.argmin == int(ix[0])
    return sol


# ---------------------------------------------------------------- walk trace


@pytest.mark.parametrize("n,k", [(1, 0), (2, 0), (2, 1), (3, 1), (5, 2), (7, 0), (8, 3),
                                 (12, 5), (13, 6), (16, 4), (18, 9)])
@pytest.mark.parametrize("kind", ["int", "float"])
def test_trace_visits_every_state_with_exact_value(n, k, kind):
    """Every x is visited exactly once and the walk's value equals Eq. 1 at it."""
    rng = np.random.default_rng(1000 * n + k)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    idx, val, sigma = qb.walk_trace(dev(Q), k)
    idx = idx.cpu().numpy().astype(np.uint64)
    val = val.cpu().numpy()
    assert np.array_equal(np.sort(idx), np.arange(1 << n, dtype=np.uint64))
    if kind == "int":
        assert sigma == 0
        assert np.array_equal(val, oracle.evaluate(Q, idx))
    else:
        # the walk is exact on round(Q * 2^sigma): compare with that image's f
        lin = np.rint(np.ldexp(np.diag(Q).astype(np.float64), sigma)).astype(np.int64)
        Qd = Q.astype(np.float64)
        S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
        Qhat = np.triu(S, 1)
        Qhat[np.diag_indices(n)] = lin
        assert np.array_equal(val, oracle.evaluate(Qhat, idx))
        f = oracle.evaluate(Q, idx)
        assert np.max(np.abs(np.ldexp(val.astype(np.float64), -sigma) - f)) <= \
            0.5 * n * (n + 1) / 2 * 2.0 ** -sigma + 1e-12


def test_trace_flip_sequence_is_binary_carry():
    """Successive states of one thread differ in bit CTZ(t) (Section 2.2's sequence)."""
    g = json.load(open(os.path.join(GOLDEN, "binary_carry.json")))
    n, k = 10, 2
    Q = np.random.default_rng(5).integers(-9, 10, size=(n, n)).astype(np.int32)
    idx, _, _ = qb.walk_trace(dev(Q), k)
    idx = idx.cpu().numpy().astype(np.int64)
    ns = n - k
    for p in range(1 << k):
        seq = idx[p << ns:(p + 1) << ns]
        assert seq[0] == p << ns
        flips = [int(np.log2(int(a) ^ int(b))) for a, b in zip(seq[:-1], seq[1:])]
        assert flips[:len(g["flip_sequence_prefix"])] == g["flip_sequence_prefix"]
        assert flips == [((t & -t).bit_length() - 1) for t in range(1, 1 << ns)]


def _fixed_point_image(Q, sigma):
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


@pytest.mark.parametrize("n,k", [(1, 0), (3, 2), (6, 0), (7, 1), (9, 3), (12, 4), (13, 2),
                                 (15, 7), (16, 10), (17, 6), (20, 8)])
@pytest.mark.parametrize("kind", ["int", "float"])
def test_min_walk_prefix_minima(n, k, kind):
    """The production MIN walk's per-prefix minima equal the oracle's, prefix by prefix."""
    rng = np.random.default_rng(77 * n + k)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.normal(size=(n, n)).astype(np.float32)
    pm, sigma = qb.prefix_minima(dev(Q), k)
    pm = pm.cpu().numpy()
    Qhat = Q.astype(np.int64) if kind == "int" else _fixed_point_image(Q, sigma)
    ns = n - k
    want = [oracle.brute_min(Qhat, p << ns, (p + 1) << ns)[0] for p in range(1 << k)]
    assert pm.tolist() == want


# ---------------------------------------------------------------- hand-worked


@pytest.mark.parametrize("name", ["hand_n2.json", "hand_n3.json"])
@pytest.mark.parametrize("dt", [np.int32, np.int16, np.float32, np.float64])
def test_hand_worked(name, dt):
    g = json.load(open(os.path.join(GOLDEN, name)))
    Q = np.array(g["Q"], dtype=dt)
    sol = qb.solve(dev(Q), top_k=3)
    assert sol.min_value == g["min"] and sol.argmin == g["argmin"]
    if "top3" in g:
        assert [[v, i] for v, i in zip(sol.topk_values, sol.topk_indices)] == g["top3"]


# ---------------------------------------------------------------- random sweeps


@pytest.mark.parametrize("n", list(range(1, 17)) + [19, 21])
def test_random_int(n):
    rng = np.random.default_rng(n)
    check_against_oracle(rng.integers(-100, 101, size=(n, n)).astype(np.int32), top_k=4)
    check_against_oracle(np.triu(rng.integers(-50, 51, size=(n, n))).astype(np.int16))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 11, 14, 17, 20])
def test_random_float(n):
    rng = np.random.default_rng(50 + n)
    check_against_oracle(np.triu(rng.uniform(-1, 1, size=(n, n))), top_k=5)
    check_against_oracle(rng.normal(size=(n, n)).astype(np.float32), top_k=2)


@pytest.mark.parametrize("k", [0, 1, 3, 5, 8, 11])
def test_prefix_width_does_not_change_answer(k):
    Q = inputs.uniform_int(14, seed=3, lo=-5, hi=5)  # many exact ties
    check_against_oracle(Q, top_k=6, prefix_bits=k)


# ---------------------------------------------------------------- workloads


def test_config_n20_f64_top8():
    """n=20 FP64 uniform[-1,1] upper, top-8: bit-exact FP64 values and indices."""
    sol = check_against_oracle(inputs.config_n20_f64(0), top_k=8)
    assert sol.n_candidates >= 8


@pytest.mark.parametrize("sparse", [False, True])
def test_config_n32_int_full(sparse):
    path = os.path.join(GOLDEN, "config_n32_int.json")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = json.load(open(path))["sparse" if sparse else "dense"]
    Q = inputs.config_n32_int(0, sparse=sparse)
    sol = qb.solve(dev(Q), top_k=8)
    assert (int(sol.min_value), sol.argmin) == (g["min"], g["argmin"])
    assert [[int(v), i] for v, i in zip(sol.topk_values, sol.topk_indices)] == g["top8"]


@pytest.mark.parametrize("sparse", [False, True])
def test_config_n32_int_sampled(sparse):
    """Full n=32 problem restricted to fixed top bits: exact against the oracle's range."""
    Q = inputs.config_n32_int(0, sparse=sparse)
    rng = np.random.default_rng(7)
    for fv in rng.integers(0, 1 << 12, size=3):
        sol = qb.solve(dev(Q), top_k=2, fix_bits=12, fix_value=int(fv))
        lo = int(fv) << 20
        vals, ix = oracle.brute_topk(Q, 2, lo, lo + (1 << 20))
        assert sol.topk_indices == [int(i) for i in ix]
        assert sol.topk_values == [float(v) for v in vals]


def test_config_n40_f32():
    """n=40 FP32: sampled sub-spaces exact; the full minimum is a verified local optimum."""
    Q = inputs.config_n40_f32(0)
    n = 40
    full = qb.solve(dev(Q))
    # value reported is the FP64 canonical value of the reported state
    assert full.min_value == oracle.evaluate(Q, full.argmin)
    # every single and double flip of the argmin is no better
    nb = [full.argmin ^ (1 << i) for i in range(n)]
    nb += [full.argmin ^ (1 << i) ^ (1 << j) for i in range(n) for j in range(i + 1, n)]
    vals = oracle.evaluate(Q, np.array(nb, dtype=np.uint64))
    assert np.all(vals >= full.min_value)
    # sub-spaces with the top 20 bits fixed (2^20 states each), including the argmin's own
    rng = np.random.default_rng(11)
    fvs = [full.argmin >> 20] + [int(v) for v in rng.integers(0, 1 << 20, size=3)]
    for fv in fvs:
        sol = qb.solve(dev(Q), fix_bits=20, fix_value=fv)
        v, am = oracle.brute_min(Q, fv << 20, (fv + 1) << 20)
        assert (sol.min_value, sol.argmin) == (v, am)
        assert full.min_value <= sol.min_value


# ---------------------------------------------------------------- edge cases


def test_edge_cases():
    # n = 1, both signs
    assert qb.solve(dev(np.array([[3]], dtype=np.int32))).argmin == 0
    s = qb.solve(dev(np.array([[-3.5]], dtype=np.float64)))
    assert (s.min_value, s.argmin) == (-3.5, 1)
    # all-zero matrices: every state ties, lowest index wins
    for dt in (np.int32, np.float32, np.float64):
        s = qb.solve(dev(np.zeros((22, 22), dtype=dt)), top_k=3)
        assert s.min_value == 0 and s.topk_indices == [0, 1, 2]
    # large all-zero matrices with top-1: exact values, only the lowest tied
    # state of each lane of the lowest prefix is re-examined
    for dt, n in ((np.float32, 30), (np.int32, 40), (np.float64, 33)):
        s = qb.solve(dev(np.zeros((n, n), dtype=dt)))
        assert (s.min_value, s.argmin) == (0, 0) and s.n_candidates <= 1 << 12
    # a variable with an all-zero row and column ties every state with its twin
    Q = inputs.uniform_int(16, seed=9)
    Q[5, :] = 0
    Q[:, 5] = 0
    check_against_oracle(Q, top_k=4)
    # diagonal closed form
    d = np.array([3, -1, 0, -7, 2, -2, 0, 5], dtype=np.int32)
    s = qb.solve(dev(np.diag(d)))
    assert s.min_value == -10 and s.argmin == (1 << 1) | (1 << 3) | (1 << 5)
    # top-k larger than the space
    s = qb.solve(dev(np.array([[1, -1], [0, -2]], dtype=np.int32)), top_k=10)
    assert s.topk_indices == [2, 3, 0, 1]


def test_errors():
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.array([[np.nan, 0], [0, 1]], dtype=np.float32)))
    assert e.value.status == qb.QBF_ENONFINITE
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.full((4, 4), 2 ** 30, dtype=np.int32)))
    assert e.value.status == qb.QBF_ERANGE
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.zeros((49, 49), dtype=np.float32)))
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.zeros((4, 4), dtype=np.int32)), top_k=65)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.zeros((4, 4), dtype=np.int32)), fix_bits=2, fix_value=4)
    assert e.value.status == qb.QBF_EINVAL
    # the library stays usable after errors
    check_against_oracle(inputs.uniform_int(10, seed=1), top_k=2)


@pytest.mark.parametrize("variant,n_ok", [(qb.QBF_VARIANT_SPLIT, 26), (qb.QBF_VARIANT_SPLIT_DEFER, 29)])
def test_block_count_limit(variant, n_ok):
    """At most 2^20 blocks of 2^6 states per thread: with prefix_bits = 0 the
    whole space is one thread's walk, allowed up to 26 suffix bits (29 for the
    eight-prefix walks, whose three group bits are not walked) and refused
    one bit beyond."""
    rng = np.random.default_rng(n_ok)
    Q = rng.normal(size=(n_ok + 1, n_ok + 1)).astype(np.float32)
    sol = qb.solve(dev(Q[:n_ok, :n_ok].copy()), prefix_bits=0, variant=variant)
    assert (sol.min_value, sol.argmin) == oracle.brute_min(Q[:n_ok, :n_ok])
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(Q), prefix_bits=0, variant=variant)
    assert e.value.status == qb.QBF_EINVAL


@pytest.mark.parametrize("n,fix", [(46, 28), (48, 34), (44, 24)])
def test_large_fix_keeps_prefix_numbers_in_range(n, fix):
    """With most variables fixed, prefix numbers pass 2^32: the automatic
    geometry would give k = 37 at n = 46, fix 28 (the planner caps it at 28),
    and fix_bits = 34 makes the prefix the fixed part itself (k = 34).  The
    flag list numbers prefixes from the sub-space's first one, so the fixed
    sub-space still matches the oracle."""
    Q = inputs.gaussian_f32(n, seed=n + fix)
    rng = np.random.default_rng(fix)
    for fv in [int(v) for v in rng.integers(0, 1 << fix, size=2)]:
        sol = qb.solve(dev(Q), fix_bits=fix, fix_value=fv)
        lo = fv << (n - fix)
        assert (sol.min_value, sol.argmin) == oracle.brute_min(Q, lo, lo + (1 << (n - fix)))
        assert sol.prefix_bits == max(28, fix)


def test_host_pointer_path_matches_device_path():
    Q = inputs.config_n20_f64(0)
    a = qb.solve(dev(Q), top_k=8)
    b = qb.solve(torch.from_numpy(Q), top_k=8)
    assert a.topk_indices == b.topk_indices and a.topk_values == b.topk_values


def test_qubo_bf_solve_one_call_form():
    """qubo_bf_solve(Q_host, n, dtype) -> min, argmin, optional top-k."""
    g = json.load(open(os.path.join(GOLDEN, "hand_n3.json")))
    Q = np.array(g["Q"], dtype=np.float64)
    v, x, top = qb.qubo_bf_solve(Q, top_k=3)
    assert (v, x) == (-2.0, 1)
    assert top == [(-2.0, 1), (-2.0, 3), (-2.0, 6)]
    Q20 = inputs.config_n20_f64(0)
    vals, ix = oracle.brute_topk(Q20, 8)
    v, x, top = qb.qubo_bf_solve(Q20, top_k=8)
    assert (v, x) == (float(vals[0]), int(ix[0]))
    assert top == [(float(a), int(b)) for a, b in zip(vals, ix)]
    Qi = np.random.default_rng(4).integers(-30, 31, size=(15, 15)).astype(np.int16)
    v, x, top = qb.qubo_bf_solve(Qi)
    ov, ox = oracle.brute_min(Qi)
    assert (v, x) == (float(ov), ox)
    assert top == []
    with pytest.raises(qb.QbfError) as e:
        qb.qubo_bf_solve(Q20, top_k=65)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.qubo_bf_solve(Q20.astype(np.uint8))
    assert e.value.status == qb.QBF_EDTYPE
