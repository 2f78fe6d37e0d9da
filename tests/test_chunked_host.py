"""Host-side logic of the chunked enumeration, with no GPU: the checkpoint
layout, merging finished shards (qbf_chunked_merge), the final result
(qbf_chunked_result), and the combine of shards held by two gloo ranks."""
import ctypes
import os
import shutil
import socket
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def qb():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2310_19373_gb300 import build

    build.build()
    from paper_2310_19373_gb300 import _binding

    return _binding


def finished_shard(qb, shard, nshards, best, top_k=4, chunk_bits=3, q_hash=0xABC, n=30):
    """A checkpoint as qbf_chunked_step leaves it after walking all chunks of
    `shard`: `best` = [(value, index), ...] of that shard."""
    ck = qb.QbfCheckpoint()
    ck.version = qb.QBF_CKPT_VERSION
    ck.n, ck.dtype, ck.top_k, ck.chunk_bits = n, 0, top_k, chunk_bits
    ck.shard, ck.nshards = shard, nshards
    ck.q_hash = q_hash
    nch = 1 << chunk_bits
    ck.chunks_done = len(range(shard, nch, nshards))
    ck.next = ck.chunks_done
    ck.done_mask = 1 << shard
    ck.n_candidates = 10 + shard
    ck.error_bound = 0.01 * (shard + 1)
    best = sorted(best)[:top_k]
    ck.count = len(best)
    for i, (v, x) in enumerate(best):
        ck.best_value[i] = v
        ck.best_index[i] = x
    return ck


def test_checkpoint_layout(qb):
    C = qb.QbfCheckpoint
    assert ctypes.sizeof(C) == 1104
    assert C.q_hash.offset == 32 and C.error_bound.offset == 72 and C.best_value.offset == 80
    assert C.best_index.offset == 80 + 8 * 64


def test_merge_orders_by_value_then_index_and_truncates(qb):
    a = finished_shard(qb, 0, 2, [(-3.0, 40), (-1.0, 7), (2.0, 9)])
    b = finished_shard(qb, 1, 2, [(-3.0, 12), (-1.0, 100), (-2.5, 5), (0.0, 1)])
    qb.qbf_chunked_merge(a, b)
    got = [(a.best_value[i], a.best_index[i]) for i in range(a.count)]
    assert got == [(-3.0, 12), (-3.0, 40), (-2.5, 5), (-1.0, 7)]
    assert a.done_mask == 3 and a.chunks_done == 8 and a.n_candidates == 21
    assert a.error_bound == 0.02
    r = qb.qbf_chunked_result(a)
    assert (r.min_value, r.argmin, r.top_k) == (-3.0, 12, 4)
    assert list(r.topk_index[:4]) == [12, 40, 5, 7]


def test_merge_and_result_refuse_bad_input(qb):
    a = finished_shard(qb, 0, 3, [(1.0, 1)])
    with pytest.raises(qb.QbfError):  # chunks of shards 1 and 2 are missing
        qb.qbf_chunked_result(a)
    for bad in (finished_shard(qb, 1, 3, [(0.0, 2)], q_hash=0xDEF),   # another Q
                finished_shard(qb, 0, 3, [(0.0, 2)]),                  # same shard
                finished_shard(qb, 1, 3, [(0.0, 2)], chunk_bits=4),    # another split
                finished_shard(qb, 1, 2, [(0.0, 2)])):                 # another shard count
        with pytest.raises(qb.QbfError) as e:
            qb.qbf_chunked_merge(a, bad)
        assert e.value.status == qb.QBF_EINVAL
    unfinished = finished_shard(qb, 1, 3, [(0.0, 2)])
    unfinished.done_mask = 0
    with pytest.raises(qb.QbfError):
        qb.qbf_chunked_merge(a, unfinished)
    old = finished_shard(qb, 1, 3, [(0.0, 2)])
    old.version = 99
    with pytest.raises(qb.QbfError):
        qb.qbf_chunked_merge(a, old)


def test_merge_is_order_independent(qb):
    lists = [[(-1.0, 3), (4.0, 8)], [(-1.0, 2), (0.5, 11)], [(-7.0, 30)]]
    outs = []
    for order in ((0, 1, 2), (2, 1, 0), (1, 2, 0)):
        cks = [finished_shard(qb, s, 3, lists[s]) for s in range(3)]
        acc = cks[order[0]]
        for s in order[1:]:
            qb.qbf_chunked_merge(acc, cks[s])
        r = qb.qbf_chunked_result(acc)
        outs.append(list(zip(r.topk_value[:r.top_k], r.topk_index[:r.top_k])))
    assert outs[0] == outs[1] == outs[2] == [(-7.0, 30), (-1.0, 2), (-1.0, 3), (0.5, 11)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2310_19373_gb300 import _binding as qb

        mine = finished_shard(qb, rank, world, [(-2.0 - rank, 100 + rank), (5.0, rank)])
        blobs = [None] * world
        dist.all_gather_object(blobs, qb.Chunked(mine).to_bytes())
        acc = qb.Chunked.from_bytes(blobs[0])
        for b in blobs[1:]:
            acc.merge(qb.Chunked.from_bytes(b))
        r = acc.result()
        out.put((rank, r.topk_values, r.topk_indices))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_their_shards(qb):
    import multiprocessing as mp

    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = ([-3.0, -2.0, 5.0, 5.0], [101, 100, 0, 1])
    assert [(r[1], r[2]) for r in res] == [want, want]
