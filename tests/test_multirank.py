"""The N > 1 host path of bench.py on CPU: two gloo ranks, replicas only.

The path has no collective: each rank solves its own copy of the instance and
the ranks meet only to take the slowest rank's time (a host all-reduce outside
the timed region).  These tests run that reduction on two real gloo processes
and check the reference arm's rank handling, with no GPU.
"""
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
if not dist.is_available():
    pytest.skip("torch.distributed is not built", allow_module_level=True)

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    pg = bench.init_ranks(world)
    try:
        ms = bench.max_over_ranks(per_rank[rank][0], pg)
        e2e = bench.max_over_ranks(per_rank[rank][1], pg)
        out.put((rank, ms, e2e, bench.replica_throughput(world, 2.0 ** 40, ms * 1e-3)))
        pg.barrier()
    finally:
        pg.destroy_process_group()


def _run_ranks(per_rank):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    world = len(per_rank)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, per_rank, out))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_two_gloo_ranks_take_the_slowest_time():
    res = _run_ranks([(83.2, 0.0841), (91.7, 0.0833)])
    assert [r[0] for r in res] == [0, 1]
    for _, ms, e2e, value in res:
        assert ms == 91.7 and e2e == 0.0841  # every rank sees the same maxima
        assert value == pytest.approx(2 * 2.0 ** 40 / 0.0917)


def test_single_process_needs_no_group():
    assert bench.init_ranks(1) is None
    assert bench.max_over_ranks(5.5, None) == 5.5
    assert bench.replica_throughput(1, 2.0 ** 40, 0.08) == 2.0 ** 40 / 0.08
    # N replicas of the same work in the same time: N times the throughput
    assert bench.replica_throughput(4, 2.0 ** 40, 0.08) == 4 * bench.replica_throughput(
        1, 2.0 ** 40, 0.08)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == b""
