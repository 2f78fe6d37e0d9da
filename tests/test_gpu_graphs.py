"""Repeated solves of the same device matrix replay a captured CUDA graph of
the solve.  The replay must read the matrix afresh, follow option changes and
report errors exactly as a direct solve does."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from conftest import ROOT
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def check(sol, Q, k):
    vals, ix = oracle.brute_topk(Q, k)
    assert sol.topk_indices == [int(i) for i in ix]
    assert sol.topk_values == [float(v) for v in vals]


@pytest.mark.parametrize("Q,k", [(inputs.gaussian_f32(18, seed=61), 3),
                                 (inputs.uniform_int(20, seed=62, lo=-9, hi=9), 2),
                                 (inputs.uniform_f64(16, seed=63), 8),
                                 (inputs.gaussian_f32(25, seed=64), 1)],
                         ids=["f32_n18", "i32_n20", "f64_n16", "f32_n25_defer"])
def test_repeated_solves_replay_and_agree(Q, k):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    for _ in range(4):  # run, capture + replay, replay, replay
        check(qb.solve(Qd, top_k=k), Q, k)


def test_replay_reads_new_contents_of_the_same_buffer():
    n = 19
    Qd = torch.from_numpy(inputs.gaussian_f32(n, seed=70)).cuda()
    for seed in range(71, 76):
        Q = inputs.gaussian_f32(n, seed=seed)
        Qd.copy_(torch.from_numpy(Q))
        check(qb.solve(Qd, top_k=2), Q, 2)


def test_replay_follows_option_changes():
    Q = inputs.gaussian_f32(17, seed=80)
    Qd = torch.from_numpy(Q).cuda()
    for _ in range(2):
        for k in (1, 5):
            for variant in (qb.QBF_VARIANT_AUTO, qb.QBF_VARIANT_SPLIT_DEFER, qb.QBF_VARIANT_SPLIT):
                s = qb.solve(Qd, top_k=k, variant=variant)
                check(s, Q, k)
                assert s.variant == (qb.QBF_VARIANT_SPLIT if variant == qb.QBF_VARIANT_AUTO
                                     else variant)
        s = qb.solve(Qd, fix_bits=3, fix_value=5)
        assert (s.min_value, s.argmin) == oracle.brute_min(Q, 5 << 14, 6 << 14)


def test_replay_reports_errors_and_recovers():
    n = 15
    Q = inputs.gaussian_f32(n, seed=90)
    Qd = torch.from_numpy(Q).cuda()
    for _ in range(3):
        check(qb.solve(Qd), Q, 1)
    bad = Q.copy()
    bad[2, 7] = np.nan
    Qd.copy_(torch.from_numpy(bad))
    with pytest.raises(qb.QbfError) as e:
        qb.solve(Qd)
    assert e.value.status == qb.QBF_ENONFINITE
    Qd.copy_(torch.from_numpy(Q))
    check(qb.solve(Qd), Q, 1)


def test_replay_can_be_switched_off():
    """QBF_NO_SOLVE_GRAPHS=1 runs every solve directly, with the same answers."""
    code = (
        "import sys, torch, numpy as np\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2310_19373_gb300 import _binding as qb, inputs\n"
        "Q = torch.from_numpy(inputs.gaussian_f32(18, seed=61)).cuda()\n"
        "for _ in range(3):\n"
        "    s = qb.solve(Q, top_k=3)\n"
        "print(s.topk_indices)\n")
    env = dict(os.environ, QBF_NO_SOLVE_GRAPHS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    _, ix = oracle.brute_topk(inputs.gaussian_f32(18, seed=61), 3)
    assert out.stdout.strip().split("\n")[-1] == str([int(i) for i in ix])
