"""GPU parity of the eight-prefix walks against the oracle: the two-pipe walk
(QBF_VARIANT_SPLIT_MIX) and the deferred-correction walk
(QBF_VARIANT_SPLIT_DEFER), which share their geometry and image bound."""
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

MIX = qb.QBF_VARIANT_SPLIT_MIX
DEFER = qb.QBF_VARIANT_SPLIT_DEFER
EIGHT = pytest.mark.parametrize("variant", [MIX, DEFER], ids=["mix", "defer"])


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def _fixed_point_image(Q, sigma):
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


# (n, k): suffix n - k = walked bits + the three group bits; walked bits <= 6
# is one unrolled block, more adds block transitions
@pytest.mark.parametrize("n,k", [(4, 0), (5, 1), (7, 0), (9, 0), (10, 1), (12, 3), (13, 0),
                                 (15, 6), (16, 9), (18, 4), (20, 7), (22, 10)])
@pytest.mark.parametrize("kind", ["int", "float"])
@EIGHT
def test_mix_prefix_minima(n, k, kind, variant):
    """Minima per prefix (k prefix bits; the eight groups of a thread are suffix bits)."""
    rng = np.random.default_rng(700 + 7 * n + k)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.normal(size=(n, n)).astype(np.float32)
    pm, sigma = qb.prefix_minima(dev(Q), k, variant)
    pm = pm.cpu().numpy()
    Qhat = Q.astype(np.int64) if kind == "int" else _fixed_point_image(Q, sigma)
    assert np.abs(np.triu(Qhat)).sum() < 2 ** 23
    ns = n - k
    want = [oracle.brute_min(Qhat, p << ns, (p + 1) << ns)[0] for p in range(1 << k)]
    assert pm.tolist() == want


@EIGHT
def test_mix_minimum_in_each_group(variant):
    """Put the unique minimum in each of the eight groups in turn (both halves
    of every packed pair, and the two int32 values of the two-pipe walk)."""
    n, k = 14, 2
    nsw = n - k - 3
    rng = np.random.default_rng(77)
    base = np.triu(rng.integers(0, 40, size=(n, n))).astype(np.int32)
    for b in range(8):
        Q = base.copy()
        # diagonal reward for exactly the group bits of b and suffix bit 0
        for t in range(3):
            Q[nsw + t, nsw + t] = -500 if (b >> t) & 1 else 500
        Q[0, 0] = -500
        pm, _ = qb.prefix_minima(dev(Q), k, variant)
        ns = n - k
        want = [oracle.brute_min(Q, p << ns, (p + 1) << ns) for p in range(1 << k)]
        assert pm.cpu().numpy().tolist() == [int(w[0]) for w in want]
        assert (want[0][1] >> nsw) & 7 == b


@pytest.mark.parametrize("n", [4, 5, 8, 11, 14, 17, 21])
@EIGHT
def test_mix_solve_against_oracle(n, variant):
    rng = np.random.default_rng(800 + n)
    for Q, k in ((rng.integers(-100, 101, size=(n, n)).astype(np.int32), 4),
                 (np.triu(rng.uniform(-1, 1, size=(n, n))), 3),
                 (rng.normal(size=(n, n)).astype(np.float32), 2)):
        sol = qb.solve(dev(Q), top_k=k, variant=variant)
        vals, ix = oracle.brute_topk(Q, k)
        assert sol.topk_indices == [int(i) for i in ix]
        assert sol.topk_values == [float(v) for v in vals]
        assert sol.variant == variant


@EIGHT
def test_mix_workloads(variant):
    g = json.load(open(os.path.join(GOLDEN, "config_n32_int.json")))["dense"]
    sol = qb.solve(dev(inputs.config_n32_int(0)), top_k=8, variant=variant)
    assert (int(sol.min_value), sol.argmin) == (g["min"], g["argmin"])
    assert [[int(v), i] for v, i in zip(sol.topk_values, sol.topk_indices)] == g["top8"]
    Q = inputs.config_n40_f32(0)
    a = qb.solve(dev(Q), variant=variant)
    b = qb.solve(dev(Q), variant=qb.QBF_VARIANT_SPLIT)
    assert (a.min_value, a.argmin) == (b.min_value, b.argmin)
    rng = np.random.default_rng(41)
    for fv in [a.argmin >> 20] + [int(v) for v in rng.integers(0, 1 << 20, size=2)]:
        s = qb.solve(dev(Q), fix_bits=20, fix_value=fv, variant=variant)
        assert (s.min_value, s.argmin) == oracle.brute_min(Q, fv << 20, (fv + 1) << 20)


@EIGHT
def test_mix_errors(variant):
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.zeros((3, 3), dtype=np.float32)), variant=variant)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.prefix_minima(dev(np.zeros((10, 10), dtype=np.float32)), 7, variant)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:  # sum |Q| >= 2^23: not exact in FP32
        qb.solve(dev(np.full((12, 12), 200000, dtype=np.int32)), variant=variant)
    assert e.value.status == qb.QBF_ERANGE


@pytest.mark.parametrize("n,k", [(12, 0), (15, 2), (19, 5)])
def test_defer_large_in_block_corrections(n, k):
    """The deferred walk keeps values without their in-block correction C[u],
    so |w| reaches |v| + |C|.  Strong couplings among the six unrolled bits
    (C up to 3e6) against strong fields of the others, with sum |Q| just
    under 2^23, still give exact minima."""
    rng = np.random.default_rng(900 + n)
    Q = np.zeros((n, n), dtype=np.int64)
    for i in range(6):
        Q[i, i] = -300000
        for j in range(i + 1, 6):
            Q[i, j] = 200000
    rest = rng.integers(-40000, 40001, size=(n, n))
    for i in range(n):
        for j in range(max(i, 6), n):
            Q[i, j] = rest[i, j]
    budget = 2 ** 23 - 2 ** 12 - np.abs(Q[:6, :6]).sum()
    tail = np.abs(Q).sum() - np.abs(Q[:6, :6]).sum()
    if tail > budget:
        Q[:, 6:] = Q[:, 6:] * budget // tail
    Q = Q.astype(np.int32)
    assert np.abs(Q.astype(np.int64)).sum() < 2 ** 23 - 2 ** 12
    pm, _ = qb.prefix_minima(dev(Q), k, DEFER)
    ns = n - k
    want = [oracle.brute_min(Q, p << ns, (p + 1) << ns)[0] for p in range(1 << k)]
    assert pm.cpu().numpy().tolist() == want
    sol = qb.solve(dev(Q), top_k=3, variant=DEFER)
    vals, ix = oracle.brute_topk(Q, 3)
    assert sol.topk_indices == [int(i) for i in ix]


def test_auto_takes_deferred_walk():
    """AUTO with n >= 24: the deferred-correction walk for float Q and for
    integer Q whose sum |Q| fits the 2^23 image; larger integer Q is repeated
    on the int32 walk."""
    n = 26
    rng = np.random.default_rng(26)
    Qf = np.triu(rng.normal(size=(n, n))).astype(np.float32)
    sol = qb.solve(dev(Qf))
    assert sol.variant == DEFER
    assert (sol.min_value, sol.argmin) == oracle.brute_min(Qf)
    Qi = np.triu(rng.integers(-50, 51, size=(n, n))).astype(np.int32)
    sol = qb.solve(dev(Qi))
    assert sol.variant == DEFER
    assert (int(sol.min_value), sol.argmin) == tuple(int(v) for v in oracle.brute_min(Qi))
    Qb = np.triu(rng.integers(-100000, 100001, size=(n, n))).astype(np.int32)
    assert np.abs(Qb.astype(np.int64)).sum() >= 2 ** 23
    for v in (MIX, DEFER):
        with pytest.raises(qb.QbfError) as e:
            qb.solve(dev(Qb), variant=v)
        assert e.value.status == qb.QBF_ERANGE
    sol = qb.solve(dev(Qb))
    assert sol.variant == qb.QBF_VARIANT_SPLIT
    assert (int(sol.min_value), sol.argmin) == tuple(int(v) for v in oracle.brute_min(Qb))
    # n < 24 stays on the int32 walk
    assert qb.solve(dev(Qf[:20, :20].copy())).variant == qb.QBF_VARIANT_SPLIT


def test_auto_falls_back_when_fp32_window_overflows():
    """One dominant entry sets the scale.  The small diagonal terms (about 0.2
    quanta of the 2^23-bounded image) round to zero there, so all 2^25 states
    with x_0 = 1 tie inside the certification window of the FP32-pipe walks,
    more candidates than the buffer holds.  In the 2^31-bounded image of the
    int32 walk they are about 55 quanta each, so AUTO repeats the solve there
    and still returns the exact optimum."""
    n = 26
    Q = np.zeros((n, n))
    Q[0, 0] = -1.0
    for i in range(1, n):
        Q[i, i] = -5e-8 * (1.0 + i / 100.0)
    for v in (MIX, DEFER, qb.QBF_VARIANT_SPLIT_F32):
        with pytest.raises(qb.QbfError) as e:
            qb.solve(dev(Q), variant=v)
        assert e.value.status == qb.QBF_EOVERFLOW
    sol = qb.solve(dev(Q))
    assert sol.variant == qb.QBF_VARIANT_SPLIT
    assert sol.argmin == (1 << n) - 1
    assert (sol.min_value, sol.argmin) == oracle.brute_min(Q)
