"""GPU parity of the packed-FP32 walk (QBF_VARIANT_SPLIT_F32) against the oracle."""
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

F32 = qb.QBF_VARIANT_SPLIT_F32


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def _fixed_point_image(Q, sigma):
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


@pytest.mark.parametrize("n,k", [(2, 0), (3, 1), (7, 0), (8, 2), (9, 5), (12, 3), (13, 0),
                                 (15, 6), (16, 9), (18, 4), (20, 7)])
@pytest.mark.parametrize("kind", ["int", "float"])
def test_f32_pair_minima(n, k, kind):
    """Minima per prefix pair (k prefix bits, n - k suffix bits incl. the pair bit)."""
    rng = np.random.default_rng(500 + 7 * n + k)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.normal(size=(n, n)).astype(np.float32)
    pm, sigma = qb.prefix_minima(dev(Q), k, F32)
    pm = pm.cpu().numpy()
    Qhat = Q.astype(np.int64) if kind == "int" else _fixed_point_image(Q, sigma)
    assert np.abs(np.triu(Qhat)).sum() < 2 ** 23
    ns = n - k
    want = [oracle.brute_min(Qhat, p << ns, (p + 1) << ns)[0] for p in range(1 << k)]
    assert pm.tolist() == want


@pytest.mark.parametrize("n", [2, 3, 5, 8, 11, 14, 17, 21])
def test_f32_solve_against_oracle(n):
    rng = np.random.default_rng(600 + n)
    for Q, k in ((rng.integers(-100, 101, size=(n, n)).astype(np.int32), 4),
                 (np.triu(rng.uniform(-1, 1, size=(n, n))), 3),
                 (rng.normal(size=(n, n)).astype(np.float32), 2)):
        sol = qb.solve(dev(Q), top_k=k, variant=F32)
        vals, ix = oracle.brute_topk(Q, k)
        assert sol.topk_indices == [int(i) for i in ix]
        assert sol.topk_values == [float(v) for v in vals]
        assert sol.variant == F32


def test_f32_workloads():
    g = json.load(open(os.path.join(GOLDEN, "config_n32_int.json")))["dense"]
    sol = qb.solve(dev(inputs.config_n32_int(0)), top_k=8, variant=F32)
    assert (int(sol.min_value), sol.argmin) == (g["min"], g["argmin"])
    assert [[int(v), i] for v, i in zip(sol.topk_values, sol.topk_indices)] == g["top8"]
    Q = inputs.config_n40_f32(0)
    a = qb.solve(dev(Q), variant=F32)
    b = qb.solve(dev(Q), variant=qb.QBF_VARIANT_SPLIT)
    assert (a.min_value, a.argmin) == (b.min_value, b.argmin)
    rng = np.random.default_rng(31)
    for fv in [a.argmin >> 20] + [int(v) for v in rng.integers(0, 1 << 20, size=2)]:
        s = qb.solve(dev(Q), fix_bits=20, fix_value=fv, variant=F32)
        assert (s.min_value, s.argmin) == oracle.brute_min(Q, fv << 20, (fv + 1) << 20)


def test_auto_takes_packed_walk_for_float_q():
    """AUTO: float Q with n >= 24 runs the packed walk, integer Q the int32 walk."""
    n = 26
    rng = np.random.default_rng(26)
    Qf = np.triu(rng.normal(size=(n, n))).astype(np.float32)
    sol = qb.solve(dev(Qf))
    assert sol.variant == F32
    assert (sol.min_value, sol.argmin) == oracle.brute_min(Qf)
    Qi = np.triu(rng.integers(-50, 51, size=(n, n))).astype(np.int32)
    sol = qb.solve(dev(Qi))
    assert sol.variant == qb.QBF_VARIANT_SPLIT
    assert (int(sol.min_value), sol.argmin) == tuple(int(v) for v in oracle.brute_min(Qi))


def test_auto_falls_back_when_packed_window_overflows():
    """One dominant entry sets the scale.  The small diagonal terms (about 0.2
    quanta of the 2^23-bounded image) round to zero there, so all 2^25 states
    with x_0 = 1 tie inside the packed walk's certification window, more
    candidates than the buffer holds.  In the 2^31-bounded image of the int32
    walk they are about 55 quanta each, so AUTO repeats the solve there and
    still returns the exact optimum."""
    n = 26
    Q = np.zeros((n, n))
    Q[0, 0] = -1.0
    for i in range(1, n):
        Q[i, i] = -5e-8 * (1.0 + i / 100.0)
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(Q), variant=F32)
    assert e.value.status == qb.QBF_EOVERFLOW
    sol = qb.solve(dev(Q))
    assert sol.variant == qb.QBF_VARIANT_SPLIT
    assert sol.argmin == (1 << n) - 1
    assert (sol.min_value, sol.argmin) == oracle.brute_min(Q)
