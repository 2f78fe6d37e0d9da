"""GPU parity of the tcgen05 blocked form (QBF_VARIANT_TC) against numpy and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402

TC = qb.QBF_VARIANT_TC


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def _fixed_point_image(Q, sigma):
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


@pytest.mark.parametrize("kind", ["integers", "fractions"])
def test_tc_single_mma_against_numpy(kind):
    """One 128x128x16 FP16 MMA through the operand layout the blocked form uses."""
    rng = np.random.default_rng(1 if kind == "integers" else 2)
    if kind == "integers":
        A = rng.integers(-2048, 2049, size=(128, 16)).astype(np.float16)
        B = rng.integers(-1024, 1025, size=(16, 128)).astype(np.float16)
    else:
        A = rng.normal(size=(128, 16)).astype(np.float16)
        B = rng.normal(size=(16, 128)).astype(np.float16)
    D = qb.qbf_tc_selftest(A.view(np.uint16), B.view(np.uint16))
    want = A.astype(np.float64) @ B.astype(np.float64)
    if kind == "integers":
        # |entries| <= 2^11 * 2^10 * 16 = 2^25: exact below 2^24 only, so compare exactly
        # where the true value is representable and closely elsewhere
        assert np.max(np.abs(D - want)) <= 4.0
        small = np.abs(want) < 2 ** 23
        assert np.array_equal(D[small], want[small])
    else:
        assert np.allclose(D, want, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("n", [15, 16, 18, 21])
@pytest.mark.parametrize("kind", ["int", "float"])
def test_tc_tile_minima(n, kind):
    """Per-tile (2^14-state) minima of the tensor-core kernel equal the oracle's."""
    rng = np.random.default_rng(300 + n)
    if kind == "int":
        Q = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    else:
        Q = rng.normal(size=(n, n)).astype(np.float32)
    k = n - 14
    pm, sigma = qb.prefix_minima(dev(Q), k, TC)
    pm = pm.cpu().numpy()
    Qhat = Q.astype(np.int64) if kind == "int" else _fixed_point_image(Q, sigma)
    # the blocked form bounds the image by 2^22
    assert np.abs(np.triu(Qhat)).sum() < 2 ** 22
    want = [oracle.brute_min(Qhat, p << 14, (p + 1) << 14)[0] for p in range(1 << k)]
    assert pm.tolist() == want


@pytest.mark.parametrize("n", [15, 17, 20, 22])
def test_tc_solve_against_oracle(n):
    rng = np.random.default_rng(n)
    for Q, k in ((rng.integers(-100, 101, size=(n, n)).astype(np.int32), 4),
                 (np.triu(rng.uniform(-1, 1, size=(n, n))), 3),
                 (rng.normal(size=(n, n)).astype(np.float32), 1)):
        sol = qb.solve(dev(Q), top_k=k, variant=TC)
        vals, ix = oracle.brute_topk(Q, k)
        assert sol.topk_indices == [int(i) for i in ix]
        assert sol.topk_values == [float(v) for v in vals]
        assert sol.variant == TC


def test_tc_config_n20_and_n32():
    Q = inputs.config_n20_f64(0)
    sol = qb.solve(dev(Q), top_k=8, variant=TC)
    vals, ix = oracle.brute_topk(Q, 8)
    assert sol.topk_indices == [int(i) for i in ix] and sol.topk_values == [float(v) for v in vals]
    Q32 = inputs.config_n32_int(0)
    a = qb.solve(dev(Q32), top_k=8, variant=TC)
    b = qb.solve(dev(Q32), top_k=8)
    assert (a.topk_values, a.topk_indices) == (b.topk_values, b.topk_indices)


def test_tc_config_n40_matches_walk_and_oracle():
    Q = inputs.config_n40_f32(0)
    tc = qb.solve(dev(Q), variant=TC)
    walk = qb.solve(dev(Q), variant=qb.QBF_VARIANT_SPLIT)
    assert (tc.min_value, tc.argmin) == (walk.min_value, walk.argmin)
    assert tc.min_value == oracle.evaluate(Q, tc.argmin)
    rng = np.random.default_rng(21)
    for fv in [tc.argmin >> 20] + [int(v) for v in rng.integers(0, 1 << 20, size=2)]:
        sol = qb.solve(dev(Q), fix_bits=20, fix_value=fv, variant=TC)
        assert (sol.min_value, sol.argmin) == oracle.brute_min(Q, fv << 20, (fv + 1) << 20)


def test_tc_rejects_out_of_range():
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.zeros((14, 14), dtype=np.float32)), variant=TC)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.solve(dev(np.full((16, 16), 30000, dtype=np.int32)), variant=TC)
    assert e.value.status == qb.QBF_ERANGE
