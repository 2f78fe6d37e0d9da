"""GPU parity of the Ising entry point (qbf_solve_ising) against direct enumeration."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402

TORCH = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i16": torch.int16}


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(TORCH[dt]).cuda()


def ising_table(J, h):
    """E(s) for every s, index i <-> s_j = 2 * bit_j(i) - 1 (FP64, direct)."""
    n = J.shape[0]
    idx = np.arange(1 << n, dtype=np.int64)
    S = 2.0 * ((idx[:, None] >> np.arange(n)) & 1) - 1.0
    Jd, hd = np.asarray(J, np.float64), np.asarray(h, np.float64)
    return np.einsum("ki,ij,kj->k", S, Jd, S) + S @ hd


def ranked(E, k):
    order = np.lexsort((np.arange(E.size), E))  # by value, then lowest index
    return E[order[:k]], order[:k]


def random_jh(rng, n, dt):
    if dt in ("i32", "i16"):
        return rng.integers(-20, 21, size=(n, n)), rng.integers(-20, 21, size=n)
    return rng.normal(size=(n, n)), rng.normal(size=n)


@pytest.mark.parametrize("dt", ["f64", "f32", "i32", "i16"])
@pytest.mark.parametrize("n", [1, 2, 5, 9, 14])
def test_ising_against_direct_enumeration(dt, n):
    rng = np.random.default_rng(900 + n)
    J, h = random_jh(rng, n, dt)
    Jt, ht = dev(J, dt), dev(h, dt)
    # the values the device sees (FP32 rounds the inputs)
    Jn, hn = Jt.double().cpu().numpy(), ht.double().cpu().numpy()
    E = ising_table(Jn, hn)
    k = min(4, 1 << n)
    vals, ix = ranked(E, k)
    sol = qb.solve_ising(Jt, ht, top_k=k)
    assert sol.topk_indices == [int(i) for i in ix]
    tol = 0.0 if dt in ("i32", "i16") else 1e-9 * (np.abs(Jn).sum() + np.abs(hn).sum())
    assert np.allclose(sol.topk_values, vals, rtol=0, atol=tol)
    assert sol.argmin == int(ix[0])
    s = np.array(sol.spins(n), dtype=np.float64)
    assert abs(s @ Jn @ s + hn @ s - sol.min_value) <= tol + 1e-12 * abs(sol.min_value)


def test_ising_fields_only():
    """J = 0: each spin opposes its field; a zero field takes s = -1 (lowest index)."""
    h = np.array([3.0, -2.0, 0.0, 0.5, -0.25, 7.0])
    sol = qb.solve_ising(dev(np.zeros((6, 6)), "f64"), dev(h, "f64"))
    assert sol.spins(6) == [-1, 1, -1, -1, 1, -1]
    assert sol.min_value == -np.abs(h).sum()


def test_ising_ferromagnet_degenerate_ground_state():
    """J_ij = -1 off the diagonal, h = 0: all-down and all-up tie; all-down
    (index 0) is returned, E = -n(n-1)."""
    n = 12
    J = -(np.ones((n, n)) - np.eye(n))
    sol = qb.solve_ising(dev(J, "i32"), dev(np.zeros(n), "i32"), top_k=2)
    assert sol.topk_indices == [0, (1 << n) - 1]
    assert sol.topk_values == [-n * (n - 1)] * 2


def test_ising_n26_against_oracle_transform():
    """Larger n: the oracle's brute force on a QUBO written out here from the
    transform (independent of the library's kernel), then E = f + c."""
    n = 26
    rng = np.random.default_rng(126)
    J, h = np.triu(rng.normal(size=(n, n)), 1), rng.normal(size=n)
    R, C = J.sum(axis=1), J.sum(axis=0)
    Q = 4 * J + np.diag(2 * h - 2 * R - 2 * C)
    c = J.sum() - h.sum()
    fmin, xmin = oracle.brute_min(Q)
    sol = qb.solve_ising(dev(J, "f64"), dev(h, "f64"))
    assert sol.argmin == xmin
    assert abs(sol.min_value - (fmin + c)) <= 1e-9 * (np.abs(J).sum() + np.abs(h).sum())


def test_ising_integer_range():
    n = 8
    J = np.full((n, n), 2 ** 29, dtype=np.int64)
    with pytest.raises(qb.QbfError) as e:
        qb.solve_ising(dev(J, "i32"), dev(np.zeros(n, dtype=np.int64), "i32"))
    assert e.value.status == qb.QBF_ERANGE
