"""Per-item parity of the batched walk at its own depth.

In the 4096-instance batched workload the n = 34 instances walk 16 suffix
bits per lane over 2^18 prefixes.  In the eight-prefix forms that is 3 group
bits and 13 walked bits: blocks of 2^6 states, mid-bit flips at levels
6..12.  qbf_solve_batched_item_minima returns the MIN pass's minimum of
every work item (32 prefixes, 2^21 states).  Each item is compared here with
the oracle's minimum of the same fixed-point image over the same natural
indices (Section 3.1's split, Algorithm 1's walk, Eq. 1's value), for every
item of one FP32 and one int16 instance, in each of the three batched walks.
"""
import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs
from test_gpu_depth import fixed_point_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402

WALKS = [(qb.QBF_VARIANT_AUTO, qb.QBF_VARIANT_SPLIT_DEFER),
         (qb.QBF_VARIANT_SPLIT_MIX, qb.QBF_VARIANT_SPLIT_MIX),
         (qb.QBF_VARIANT_SPLIT, qb.QBF_VARIANT_SPLIT)]


@pytest.fixture(scope="module")
def batch():
    Qs = inputs.config_batched()
    dev = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in Qs]
    f34 = next(i for i, q in enumerate(Qs) if q.shape[0] == 34 and q.dtype == np.float32)
    i34 = next(i for i, q in enumerate(Qs) if q.shape[0] == 34 and q.dtype == np.int16)
    return Qs, dev, (f34, i34)


@pytest.mark.parametrize("variant,walk", WALKS, ids=["auto-defer", "mix", "split"])
def test_every_item_of_the_n34_instances_equals_oracle(batch, variant, walk):
    Qs, dev, picks = batch
    for inst in picks:
        n = Qs[inst].shape[0]
        # the default width, explicitly: a tuner run earlier in the process
        # may have changed the process-wide default
        mins, nit, info = qb.batched_item_minima(dev, inst, 1 << 16, batch_suffix_bits=16,
                                                 variant=variant)
        inf = info[inst]
        assert inf.walk == walk
        s = inf.suffix_bits
        assert inf.prefix_bits == n - s
        assert nit == (1 << (n - s)) // 32 and len(mins) == nit
        Qhat = fixed_point_image(Qs[inst], inf.scale_bits)
        want, _ = oracle.segment_minima(Qhat, 32 << s, nit)
        got = np.asarray(mins, dtype=np.int64)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (inst, variant, bad[:8], got[bad[:8]], want[bad[:8]])


def test_item_minima_errors(batch):
    Qs, dev, _ = batch
    small = dev[:4]
    for bad in (4, -1):
        with pytest.raises(qb.QbfError) as e:
            qb.batched_item_minima(small, bad, 16)
        assert e.value.status == qb.QBF_EINVAL
    # max_items = 0 only reports the count
    mins, nit, info = qb.batched_item_minima(small, 0, 0)
    assert mins == [] and nit == max(1, (1 << info[0].prefix_bits) // 32)
