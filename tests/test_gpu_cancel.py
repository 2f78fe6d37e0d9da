"""qbf_cancel: another host thread stops the running solve.

The walks read the cancellation word whenever a warp takes a work item, so a
long solve returns QBF_ECANCELED well before its end, and the next call,
which clears the word when it starts, runs to a correct answer.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def dev(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def test_cancel_stops_a_long_solve_and_the_next_one_runs():
    small = inputs.gaussian_f32(20, seed=2)
    qb.solve(dev(small))  # library loaded, pools built
    Q = dev(inputs.gaussian_f32(44, seed=7))  # 2^44 states: about 0.85 s uncancelled
    torch.cuda.synchronize()
    timer = threading.Timer(0.15, qb.qbf_cancel)
    t0 = time.perf_counter()
    timer.start()
    with pytest.raises(qb.QbfError) as e:
        qb.solve(Q)
    dt = time.perf_counter() - t0
    timer.join()
    assert e.value.status == qb.QBF_ECANCELED
    assert dt < 0.6, dt
    s = qb.solve(dev(small))
    assert (s.min_value, s.argmin) == oracle.brute_min(small)


def test_cancel_with_nothing_running_has_no_effect():
    qb.qbf_cancel()
    Q = inputs.gaussian_f32(18, seed=3)
    s = qb.solve(dev(Q))
    assert (s.min_value, s.argmin) == oracle.brute_min(Q)


def test_cancel_stops_a_batched_solve():
    Qs = [dev(q) for q in inputs.config_batched()]  # about 0.39 s uncancelled
    small = [dev(inputs.gaussian_f32(16, seed=s)) for s in range(3)]
    qb.solve_batched(small)
    torch.cuda.synchronize()
    timer = threading.Timer(0.08, qb.qbf_cancel)
    t0 = time.perf_counter()
    timer.start()
    with pytest.raises(qb.QbfError) as e:
        qb.solve_batched(Qs)
    dt = time.perf_counter() - t0
    timer.join()
    assert e.value.status == qb.QBF_ECANCELED
    assert dt < 0.3, dt
    vmin, am = qb.solve_batched(small)
    for q, v, a in zip(small, vmin, am):
        assert (v, a) == oracle.brute_min(q.cpu().numpy())


def test_release_frees_the_words_and_the_next_calls_rebuild_them():
    small = inputs.gaussian_f32(20, seed=4)
    qb.solve(dev(small))
    qb.qbf_release()  # pools, graphs and cancellation words freed
    s = qb.solve(dev(small))
    assert (s.min_value, s.argmin) == oracle.brute_min(small)
    Q = dev(inputs.gaussian_f32(44, seed=8))
    torch.cuda.synchronize()
    timer = threading.Timer(0.15, qb.qbf_cancel)
    t0 = time.perf_counter()
    timer.start()
    with pytest.raises(qb.QbfError) as e:
        qb.solve(Q)
    dt = time.perf_counter() - t0
    timer.join()
    assert e.value.status == qb.QBF_ECANCELED
    assert dt < 0.6, dt
