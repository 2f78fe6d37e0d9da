"""Per-prefix parity at the full walk depth of the n = 40 solve.

A certified n = 40 solve walks 16 suffix bits per lane for 2^21 prefixes: the
table-driven deferred walk in blocks of 2^7 states (mid-bit flips at levels
7..15), the record-driven walks in blocks of 2^6 (records at levels 6..15).  Walking all of
them against the oracle is too slow for a test, so qbf_prefix_minima_fixed
runs the production MIN kernel in exactly that geometry over windows of 2^11
prefixes (the top prefix variables fixed), and every prefix's minimum of the
fixed-point image round(Q * 2^sigma) is compared with the oracle's minimum
over the same 2^(n - prefix_bits) natural indices (Section 3.1's split,
Algorithm 1's walk, Eq. 1's value).
"""
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


def fixed_point_image(Q, sigma):
    """round(Q * 2^sigma) as the walks take it: lin on the diagonal, the
    symmetrised off-diagonal S_ij = Q_ij + Q_ji above it (round half to even)."""
    Qd = np.asarray(Q, dtype=np.float64)
    n = Qd.shape[0]
    S = np.rint(np.ldexp(Qd + Qd.T, sigma)).astype(np.int64)
    Qhat = np.triu(S, 1)
    Qhat[np.diag_indices(n)] = np.rint(np.ldexp(np.diag(Qd), sigma)).astype(np.int64)
    return Qhat


# (variant, prefix_bits of the automatic n = 40 geometry): suffix = 19 for the
# eight-prefix walks (16 walked + 3 group bits), 17 for the packed pair walk
# (16 + 1 pair bit), 16 for the int32 walk, 14 (one tile) for the tensor-core form;
# and the table-driven deferred walk at the two lane depths around its switch
# from 128-step to 64-step blocks (14 walked bits: 2^7 blocks of 128; 13: 2^7
# blocks of 64)
FORMS = [(qb.QBF_VARIANT_SPLIT_DEFER, 21), (qb.QBF_VARIANT_SPLIT_MIX, 21),
         (qb.QBF_VARIANT_SPLIT_F32, 23), (qb.QBF_VARIANT_SPLIT, 24), (qb.QBF_VARIANT_TC, 26),
         (qb.QBF_VARIANT_SPLIT_DEFER, 23), (qb.QBF_VARIANT_SPLIT_DEFER, 24)]
WINDOW = 11  # prefixes per window: 2^11


@pytest.mark.parametrize("variant,k", FORMS,
                         ids=["defer", "mix", "f32", "split", "tc", "defer-14", "defer-13"])
def test_n40_prefix_minima_at_full_depth(variant, k):
    n = 40
    Q = inputs.config_n40_f32(0)
    g = json.load(open(os.path.join(GOLDEN, "config_n40_f32.json")))
    fix = k - WINDOW
    ns = n - k
    rng = np.random.default_rng(4040 + variant)
    windows = [0, (1 << fix) - 1, g["argmin"] >> (n - fix), int(rng.integers(1, (1 << fix) - 1))]
    Qd = torch.from_numpy(Q).cuda()
    for fv in windows:
        pm, sigma = qb.prefix_minima_fixed(Qd, k, fix, fv, variant)
        Qhat = fixed_point_image(Q, sigma)
        want, _ = oracle.segment_minima(Qhat, 1 << ns, 1 << WINDOW, lo=fv << (n - fix))
        got = pm.cpu().numpy().astype(np.int64)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (fv, bad[:5], got[bad[:5]], want[bad[:5]])


def test_prefix_minima_fixed_errors():
    Qd = torch.from_numpy(inputs.gaussian_f32(20, seed=1)).cuda()
    pm = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(qb.QbfError) as e:  # more fixed bits than prefix bits
        qb.qbf_prefix_minima_fixed(Qd.data_ptr(), 20, qb.QBF_F32, 8, qb.QBF_VARIANT_SPLIT, 9, 0,
                                   pm.data_ptr())
    assert e.value.status == qb.QBF_EINVAL
    with pytest.raises(qb.QbfError) as e:  # fix_value wider than fix_bits
        qb.qbf_prefix_minima_fixed(Qd.data_ptr(), 20, qb.QBF_F32, 8, qb.QBF_VARIANT_SPLIT, 6,
                                   1 << 6, pm.data_ptr())
    assert e.value.status == qb.QBF_EINVAL


@pytest.mark.parametrize("variant", [qb.QBF_VARIANT_SPLIT, qb.QBF_VARIANT_SPLIT_DEFER])
def test_prefix_minima_fixed_matches_whole_space_run(variant):
    """The window run gives the same minima as the slice of a whole-space run."""
    n, k, fix = 22, 10, 3
    Q = inputs.gaussian_f32(n, seed=9)
    Qd = torch.from_numpy(Q).cuda()
    full, s1 = qb.prefix_minima(Qd, k, variant)
    for fv in range(1 << fix):
        part, s2 = qb.prefix_minima_fixed(Qd, k, fix, fv, variant)
        assert s1 == s2
        w = 1 << (k - fix)
        assert np.array_equal(part.cpu().numpy(), full.cpu().numpy()[fv * w:(fv + 1) * w])


@pytest.mark.parametrize("variant", [qb.QBF_VARIANT_SPLIT_DEFER, qb.QBF_VARIANT_AUTO])
def test_deep_suffix_takes_the_record_driven_walk(variant):
    """A lane walking more than 2^14 blocks (here 2^15: 21 walked bits) does not
    fit the table-driven form's suffix table and runs the record-driven
    deferred walk; its per-prefix minima and the solve still equal the oracle."""
    n, k = 26, 2  # suffix 24 = 3 group bits + 21 walked bits
    Q = inputs.gaussian_f32(n, seed=26)
    Qd = torch.from_numpy(Q).cuda()
    pm, sigma = qb.prefix_minima(Qd, k, qb.QBF_VARIANT_SPLIT_DEFER)
    want, _ = oracle.segment_minima(fixed_point_image(Q, sigma), 1 << (n - k), 1 << k)
    assert np.array_equal(pm.cpu().numpy().astype(np.int64), want)
    s = qb.solve(Qd, variant=variant, prefix_bits=k)
    assert (s.min_value, s.argmin) == oracle.blocked_min(Q)
