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

