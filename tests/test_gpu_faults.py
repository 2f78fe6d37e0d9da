"""Host-side fault injection: error paths that need no GPU fault.

With QBF_INJECT_ALLOC_FAILURE set, a scratch pool that has to grow reports a
failed allocation.  The calls must return QBF_ECUDA with a message naming
the injection, leave the process usable, and solve correctly once the
variable is gone.  The run is a fresh process, so its pools start empty.
"""
import os
import subprocess
import sys

import pytest

import oracle
from conftest import ROOT
from paper_2310_19373_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_injected_allocation_failure_is_reported_and_recoverable():
    code = (
        "import os, sys, torch\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2310_19373_gb300 import _binding as qb, inputs\n"
        "Q = torch.from_numpy(inputs.gaussian_f32(26, seed=1)).cuda()\n"
        "os.environ['QBF_INJECT_ALLOC_FAILURE'] = '1'\n"
        "for call in (lambda: qb.solve(Q), lambda: qb.solve_batched([Q])):\n"
        "    try:\n"
        "        call()\n"
        "        print('no error')\n"
        "    except qb.QbfError as e:\n"
        "        print(e.status, 'injected' in str(e))\n"
        "del os.environ['QBF_INJECT_ALLOC_FAILURE']\n"
        "s = qb.solve(Q)\n"
        "v, a = qb.solve_batched([Q])\n"
        "print(s.min_value, s.argmin, v[0], a[0])\n")
    env = {k: v for k, v in os.environ.items() if k != "QBF_INJECT_ALLOC_FAILURE"}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().split("\n")[-3:]
    from paper_2310_19373_gb300 import _binding as qb
    assert lines[0] == f"{qb.QBF_ECUDA} True"
    assert lines[1] == f"{qb.QBF_ECUDA} True"
    v1, a1, v2, a2 = lines[2].split()
    want = oracle.brute_min(inputs.gaussian_f32(26, seed=1))
    assert (float(v1), int(a1)) == want
    assert (float(v2), int(a2)) == want
