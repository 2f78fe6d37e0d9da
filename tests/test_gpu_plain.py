"""GPU parity of the two reference forms: the plain Gray walk with a per-thread
field vector (QBF_VARIANT_FIELD) and the naive natural-order evaluator
(QBF_VARIANT_NAIVE), against the oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402

FIELD, NAIVE = qb.QBF_VARIANT_FIELD, qb.QBF_VARIANT_NAIVE


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def _fixed_point_image(Q, sigma):
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


@pytest.mark.parametrize("variant", [FIELD, NAIVE])
@pytest.mark.parametrize("n,k", [(1, 0), (2, 1), (5, 0), (9, 3), (13, 5), (17, 4), (22, 2)])
@pytest.mark.parametrize("kind", ["int", "float"])
def test_plain_prefix_minima(variant, n, k, kind):
    rng = np.random.default_rng(1000 + 7 * n + k)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.normal(size=(n, n)).astype(np.float32)
    pm, sigma = qb.prefix_minima(dev(Q), k, variant)
    Qhat = Q.astype(np.int64) if kind == "int" else _fixed_point_image(Q, sigma)
    ns = n - k
    want = [oracle.brute_min(Qhat, p << ns, (p + 1) << ns)[0] for p in range(1 << k)]
    assert pm.cpu().numpy().tolist() == want


@pytest.mark.parametrize("variant", [FIELD, NAIVE])
@pytest.mark.parametrize("n", [3, 8, 14, 19])
def test_plain_solve_against_oracle(variant, n):
    rng = np.random.default_rng(1100 + n)
    for Q, k in ((rng.integers(-100, 101, size=(n, n)).astype(np.int32), 4),
                 (np.triu(rng.uniform(-1, 1, size=(n, n))), 3),
                 (rng.normal(size=(n, n)).astype(np.float32), 2)):
        sol = qb.solve(dev(Q), top_k=k, variant=variant)
        vals, ix = oracle.brute_topk(Q, k)
        assert sol.topk_indices == [int(i) for i in ix]
        assert sol.topk_values == [float(v) for v in vals]
        assert sol.variant == variant


def test_plain_forms_agree_with_split_walk_n28():
    Q = np.triu(np.random.default_rng(28).normal(size=(28, 28))).astype(np.float32)
    ref = qb.solve(dev(Q), variant=qb.QBF_VARIANT_SPLIT)
    for v in (FIELD, NAIVE):
        sol = qb.solve(dev(Q), variant=v)
        assert (sol.min_value, sol.argmin) == (ref.min_value, ref.argmin)


def test_field_suffix_limit():
    Q = dev(np.zeros((24, 24), dtype=np.float32))
    with pytest.raises(qb.QbfError) as e:
        qb.prefix_minima(Q, 3, FIELD)  # 21 suffix bits
    assert e.value.status == qb.QBF_EINVAL
    pm, _ = qb.prefix_minima(Q, 4, FIELD)  # 20 suffix bits: allowed
    assert pm.cpu().numpy().tolist() == [0] * 16
