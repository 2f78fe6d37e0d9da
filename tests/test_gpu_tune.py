"""The batched solver's autotuner (qbf_tune), its cache file, and the
per-instance certification details (qbf_solve_batched_info)."""
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


def to_dev(Qs):
    return [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in Qs]


def device_tag():
    p = torch.cuda.get_device_properties(0)
    return p.name.replace(" ", "_"), p.multi_processor_count


def test_tune_cache_then_solve(tmp_path):
    """qbf_tune picks (suffix width, CTAs per SM) for each n, appends one cache
    line per n, takes effect at once, and the solve that uses it still gives
    the oracle's answers."""
    path = str(tmp_path / "tune.txt")
    qb.qbf_tune(20, 23, qb.QBF_F32, path)
    qb.qbf_tune(21, 21, qb.QBF_I16, path)
    lines = open(path).read().split("\n")
    lines = [ln.split() for ln in lines if ln]
    assert len(lines) == 5
    name, nsm = device_tag()
    for ln in lines:
        assert ln[0] == "qbf-tune-v1" and ln[1] == name and int(ln[2]) == nsm
        assert 6 <= int(ln[5]) <= 18 and int(ln[6]) >= 1 and float(ln[7]) > 0
    want = {(int(ln[3]), int(ln[4])): (int(ln[5]), int(ln[6])) for ln in lines}
    for n in range(20, 24):
        assert qb.qbf_tuned_params(n, qb.QBF_F32) == want[(0, n)]
    assert qb.qbf_tuned_params(21, qb.QBF_I16) == want[(1, 21)]
    Qs = [inputs.gaussian_f32(n, seed=n) for n in (20, 21, 22, 23)]
    Qs += [inputs.uniform_int(21, seed=5, lo=-50, hi=50, dtype=np.int16)]
    vmin, am, info = qb.solve_batched_info(to_dev(Qs))
    for i, Q in enumerate(Qs):
        assert (vmin[i], am[i]) == oracle.brute_min(Q), i
        n = Q.shape[0]
        cls = 1 if Q.dtype == np.int16 else 0
        assert info[i].suffix_bits == max(6, min(want[(cls, n)][0], max(n, 11) - 5))


def test_cache_is_loaded_by_a_fresh_process(tmp_path):
    """A process whose first batched call finds a cache line for its device uses
    that suffix width (QBF_TUNE_CACHE names the default cache)."""
    name, nsm = device_tag()
    path = tmp_path / "cache.txt"
    path.write_text(f"qbf-tune-v1 {name} {nsm} 0 24 9 2 0.001\n"
                    f"qbf-tune-v1 other_device 7 0 24 12 1 0.001\n")
    code = (
        "import numpy as np, torch, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2310_19373_gb300 import _binding as qb, inputs\n"
        "print(qb.qbf_tuned_params(24, qb.QBF_F32))\n"
        "Q = torch.from_numpy(inputs.gaussian_f32(24, seed=1)).cuda()\n"
        "v, a, info = qb.solve_batched_info([Q])\n"
        "print(info[0].suffix_bits, info[0].prefix_bits, v[0], a[0])\n")
    env = dict(os.environ, QBF_TUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    l1, l2 = out.stdout.strip().split("\n")[-2:]
    assert l1 == "(9, 2)"
    ns, k, v, a = l2.split()
    assert (int(ns), int(k)) == (9, 15)
    assert (float(v), int(a)) == oracle.brute_min(inputs.gaussian_f32(24, seed=1))


def test_batched_info_fields():
    """Per-instance details: integer instances certify with a zero window, float
    ones with the same sigma and window as the single-instance deferred walk;
    at least one state is rescored per instance; the walk form is named."""
    Qs = [inputs.gaussian_f32(18, seed=1), inputs.uniform_f64(22, seed=2),
          inputs.uniform_int(20, seed=3, lo=-50, hi=50, dtype=np.int16),
          inputs.uniform_int(14, seed=4, lo=-9, hi=9, dtype=np.int32)]
    vmin, am, info = qb.solve_batched_info(to_dev(Qs))
    for i, Q in enumerate(Qs):
        assert (vmin[i], am[i]) == oracle.brute_min(Q)
        assert info[i].n_candidates >= 1
        assert info[i].walk in (qb.QBF_VARIANT_SPLIT_DEFER, qb.QBF_VARIANT_SPLIT)
        assert info[i].suffix_bits + info[i].prefix_bits == max(Q.shape[0], 11)
    assert info[2].error_bound == 0 and info[3].error_bound == 0
    for i in (0, 1):
        s = qb.solve(torch.from_numpy(Qs[i]).cuda(), variant=qb.QBF_VARIANT_SPLIT_DEFER)
        assert info[i].scale_bits == s.scale_bits
        assert info[i].error_bound == s.error_bound
    # the int32 pass names its walk
    _, _, info2 = qb.solve_batched_info(to_dev(Qs), variant=qb.QBF_VARIANT_SPLIT)
    assert all(x.walk == qb.QBF_VARIANT_SPLIT for x in info2)


def test_tune_errors():
    with pytest.raises(qb.QbfError) as e:
        qb.qbf_tune(30, 20, qb.QBF_F32)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.qbf_tune(20, 35, qb.QBF_F32)
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:
        qb.qbf_tune(20, 21, 9)
    assert e.value.status == qb.QBF_EDTYPE
