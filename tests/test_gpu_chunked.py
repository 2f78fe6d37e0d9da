"""GPU parity of the chunked, resumable enumeration against qbf_solve and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def same(sol, ref):
    assert sol.topk_indices == ref.topk_indices
    assert sol.topk_values == ref.topk_values


def test_resume_from_bytes_after_every_step():
    Q = dev(inputs.gaussian_f32(30, seed=3))
    ref = qb.solve(Q, top_k=4)
    blob = qb.Chunked.start(Q, chunk_bits=5, top_k=4).to_bytes()
    steps = 0
    while True:
        c = qb.Chunked.from_bytes(blob)  # a fresh process would do the same
        done = c.step(Q, max_chunks=3)
        blob = c.to_bytes()
        steps += 1
        if done:
            break
    assert steps == 11  # 32 chunks, 3 per step
    c = qb.Chunked.from_bytes(blob)
    assert c.ck.chunks_done == 32
    same(c.result(), ref)


def test_integer_q_exact():
    Qn = np.triu(np.random.default_rng(8).integers(-100, 101, size=(28, 28))).astype(np.int32)
    Q = dev(Qn)
    c = qb.Chunked.start(Q, chunk_bits=4, top_k=3)
    assert c.step(Q, max_chunks=1 << 20)
    r = c.result()
    vals, ix = oracle.brute_topk(Qn, 3)
    assert r.topk_indices == [int(i) for i in ix] and r.topk_values == [float(v) for v in vals]
    assert r.error_bound == 0.0


@pytest.mark.parametrize("nshards", [3, 5])
def test_shards_merge_to_the_whole(nshards):
    Q = dev(inputs.gaussian_f32(27, seed=5))
    ref = qb.solve(Q, top_k=5)
    parts = []
    for r in range(nshards):
        c = qb.Chunked.start(Q, chunk_bits=2, top_k=5, shard=r, nshards=nshards)
        while not c.step(Q, max_chunks=1):
            pass
        parts.append(c)
    acc = parts[-1]
    for c in parts[:-1]:
        acc.merge(c)
    same(acc.result(), ref)


def test_two_states_per_chunk_against_oracle():
    Qn = np.random.default_rng(10).normal(size=(10, 10))
    Q = dev(Qn)
    c = qb.Chunked.start(Q, chunk_bits=9, top_k=6)
    c.step(Q, max_chunks=1 << 9)
    r = c.result()
    vals, ix = oracle.brute_topk(Qn, 6)
    assert r.topk_indices == [int(i) for i in ix] and r.topk_values == [float(v) for v in vals]


def test_step_refuses_another_q():
    Q = dev(inputs.gaussian_f32(24, seed=1))
    c = qb.Chunked.start(Q, chunk_bits=3)
    c.step(Q, max_chunks=2)
    other = dev(inputs.gaussian_f32(24, seed=2))
    with pytest.raises(qb.QbfError) as e:
        c.step(other, max_chunks=2)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError):
        c.result()  # unfinished


def test_n44_chunked_properties_and_sampled_ranges():
    """n = 44 (beyond one launch's comfortable size): the certified minimum of
    the chunked run is the oracle's value of the returned state, it is no
    larger than any sampled 2^20-state range's minimum, and those ranges,
    solved on the GPU, match the oracle exactly."""
    n = 44
    Qn = inputs.gaussian_f32(n, seed=44)
    Q = dev(Qn)
    c = qb.Chunked.start(Q, chunk_bits=4, top_k=2)
    assert c.step(Q, max_chunks=16)
    r = c.result()
    assert r.min_value == oracle.evaluate(Qn, r.argmin)
    assert r.topk_values[1] == oracle.evaluate(Qn, r.topk_indices[1])
    assert (r.topk_values[0], r.topk_indices[0]) < (r.topk_values[1], r.topk_indices[1])
    rng = np.random.default_rng(144)
    for fv in [r.argmin >> 20] + [int(v) for v in rng.integers(0, 1 << 24, size=3)]:
        s = qb.solve(Q, fix_bits=24, fix_value=fv)
        want = oracle.brute_min(Qn, fv << 20, (fv + 1) << 20)
        assert (s.min_value, s.argmin) == want
        assert r.min_value <= s.min_value
