"""GPU parity of the batched persistent solver (qbf_solve_batched) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def to_dev(Qs):
    return [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in Qs]


def test_batched_small_mixed_against_oracle():
    rng = np.random.default_rng(0)
    Qs = []
    for i in range(96):
        n = int(rng.integers(1, 19))
        kind = i % 4
        if kind == 0:
            Qs.append(np.triu(rng.uniform(-1, 1, size=(n, n))).astype(np.float32))
        elif kind == 1:
            Qs.append(rng.integers(-50, 51, size=(n, n)).astype(np.int16))
        elif kind == 2:
            Qs.append(rng.normal(size=(n, n)))  # float64, not triangular
        else:
            Qs.append(np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.int32))  # many ties
    vmin, am = qb.solve_batched(to_dev(Qs))
    for i, Q in enumerate(Qs):
        v, a = oracle.brute_min(Q)
        assert (vmin[i], am[i]) == (float(v), a), i


@pytest.mark.parametrize("bits", [6, 9, 14, 16, 18])
def test_batched_suffix_width_does_not_change_answer(bits):
    Qs = [inputs.uniform_int(int(n), seed=int(n), lo=-5, hi=5) for n in (11, 14, 17, 20, 22)]
    Qs += [inputs.gaussian_f32(int(n), seed=int(n)) for n in (12, 19, 21)]
    vmin, am = qb.solve_batched(to_dev(Qs), batch_suffix_bits=bits)
    for i, Q in enumerate(Qs):
        v, a = oracle.brute_min(Q)
        assert (vmin[i], am[i]) == (float(v), a), (bits, i)


def test_batched_degenerate_instances():
    Qs = [np.zeros((20, 20), dtype=np.float32), np.zeros((13, 13), dtype=np.int32),
          np.array([[-2.0]]), np.array([[5]], dtype=np.int16), np.diag([1.0, -1.0, 0.0, -3.0])]
    vmin, am = qb.solve_batched(to_dev(Qs))
    assert (vmin[0], am[0]) == (0.0, 0)
    assert (vmin[1], am[1]) == (0.0, 0)
    assert (vmin[2], am[2]) == (-2.0, 1)
    assert (vmin[3], am[3]) == (0.0, 0)
    assert (vmin[4], am[4]) == (-4.0, 0b1010)


def test_batched_errors():
    with pytest.raises(qb.QbfError) as e:
        qb.solve_batched(to_dev([np.zeros((35, 35), dtype=np.float32)]))
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.solve_batched(to_dev([np.eye(4, dtype=np.float32), np.full((3, 3), np.inf,
                                                                      dtype=np.float32)]))
    assert e.value.status == qb.QBF_ENONFINITE and "instance 1" in str(e.value)


def test_batched_config_4096():
    """The 4096-instance workload (n ~ U{16..34}, half FP32, half int16) in one call."""
    Qs = inputs.config_batched()
    vmin, am = qb.solve_batched(to_dev(Qs))
    ns = np.array([q.shape[0] for q in Qs])
    # every reported value is the oracle's value of the reported state, and no
    # single flip improves it
    for i, Q in enumerate(Qs):
        n = Q.shape[0]
        assert vmin[i] == oracle.evaluate(Q, am[i]), i
        nb = np.array([am[i] ^ (1 << b) for b in range(n)], dtype=np.uint64)
        assert np.all(oracle.evaluate(Q, nb) >= vmin[i]), i
        assert am[i] < (1 << n)
    # exact against the oracle: every instance with n <= 20, and a sample up to n = 25
    rng = np.random.default_rng(3)
    small = [i for i in range(len(Qs)) if ns[i] <= 20]
    mid = list(rng.choice([i for i in range(len(Qs)) if 21 <= ns[i] <= 25], size=6,
                          replace=False))
    for i in small + mid:
        v, a = oracle.brute_min(Qs[i])
        assert (vmin[i], am[i]) == (float(v), a), i
    # the largest instances (n >= 32, too large to enumerate here): the 2^20-state
    # window of natural indices around the reported argmin gives exactly
    # (min, argmin), and two random windows do no better
    big = [i for i in range(len(Qs)) if ns[i] >= 32][:12]
    for i in big:
        lo = (am[i] >> 20) << 20
        v, a = oracle.brute_min(Qs[i], lo, lo + (1 << 20))
        assert (vmin[i], am[i]) == (float(v), a), i
        for w in rng.integers(0, 1 << (int(ns[i]) - 20), size=2):
            v, _ = oracle.brute_min(Qs[i], int(w) << 20, (int(w) + 1) << 20)
            assert float(v) >= vmin[i], i


def test_batched_tuner_and_repeat():
    Qs = [inputs.uniform_int(int(n), seed=int(n)) for n in range(16, 27)]
    dQs = to_dev(Qs)
    ptrs = [q.data_ptr() for q in dQs]
    stream = torch.cuda.current_stream().cuda_stream
    best, sec = qb.qbf_tune_batched(ptrs, [q.shape[0] for q in Qs], [qb.QBF_I32] * len(Qs), 10,
                                    15, stream)
    assert 10 <= best <= 15 and sec > 0
    first = qb.solve_batched(dQs)
    second = qb.solve_batched(dQs)  # graph replay
    assert first == second
    for i, Q in enumerate(Qs):
        v, a = oracle.brute_min(Q)
        assert (first[0][i], first[1][i]) == (float(v), a)


@pytest.mark.parametrize("variant", [qb.QBF_VARIANT_AUTO, qb.QBF_VARIANT_SPLIT_DEFER,
                                     qb.QBF_VARIANT_SPLIT_MIX], ids=["auto", "defer", "mix"])
def test_batched_eight_prefix_pass_matches_int32_pass(variant):
    """AUTO and SPLIT_DEFER (the deferred-correction MIN walk for instances
    whose image fits 2^23), SPLIT_MIX (the two-pipe walk there) and
    QBF_VARIANT_SPLIT (the int32 walk throughout) certify the same answers on
    a mixed batch: FP32/FP64 and integer instances, small n (int32 walk inside
    the FP32-image pass) and large n, and an integer instance too large for
    the 2^23 image."""
    rng = np.random.default_rng(77)
    Qs = []
    for i, n in enumerate([12, 16, 19, 22, 24, 26, 27, 25, 23, 20]):
        if i % 3 == 0:
            Qs.append(rng.integers(-50, 51, size=(n, n)).astype(np.int16))
        elif i % 3 == 1:
            Qs.append(rng.normal(size=(n, n)).astype(np.float32))
        else:
            Qs.append(np.triu(rng.uniform(-1, 1, size=(n, n))))
    big = np.triu(rng.integers(-100000, 100001, size=(24, 24))).astype(np.int32)
    assert np.abs(big.astype(np.int64)).sum() >= 2 ** 23
    Qs.append(big)
    dQs = to_dev(Qs)
    a = qb.solve_batched(dQs, variant=variant)
    b = qb.solve_batched(dQs, variant=qb.QBF_VARIANT_SPLIT)
    assert a == b
    for Q, v, x in zip(Qs, *a):
        ov, ox = oracle.brute_min(Q)
        assert (v, x) == (float(ov), ox)


def test_batched_auto_falls_back_when_fp32_windows_overflow():
    """The instance of tests/test_gpu_mix.py whose small terms vanish in the
    2^23 image (2^25 states inside the window) overflows the batch's
    candidate buffer on the FP32-image passes; AUTO repeats the batch on the int32
    pass and still certifies every instance."""
    n = 26
    Q = np.zeros((n, n))
    Q[0, 0] = -1.0
    for i in range(1, n):
        Q[i, i] = -5e-8 * (1.0 + i / 100.0)
    other = np.random.default_rng(3).normal(size=(20, 20)).astype(np.float32)
    dQs = to_dev([other, Q])
    for v in (qb.QBF_VARIANT_SPLIT_MIX, qb.QBF_VARIANT_SPLIT_DEFER):
        with pytest.raises(qb.QbfError) as e:
            qb.solve_batched(dQs, variant=v)
        assert e.value.status == qb.QBF_EOVERFLOW
    vmin, am = qb.solve_batched(dQs)
    assert (vmin[1], am[1]) == oracle.brute_min(Q)
    assert am[1] == (1 << n) - 1
    assert (vmin[0], am[0]) == oracle.brute_min(other)
