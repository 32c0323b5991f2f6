"""The multi-rank path of the benchmark on CPU: two gloo ranks (127.0.0.1)
take disjoint ensemble members and their own seeds, and reduce timings with
the maximum over ranks; throughput counts both ranks' units over the slowest
rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2001_01624_gb300 import replicas as R  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        members = R.member_indices(rank, 5)
        t = R.max_over_ranks(dist, [10.0 * (rank + 1), 3.0 - rank], "cpu")
        dist.barrier()
        q.put((rank, members, R.geomodel_seed(rank), R.serving_seed(rank), t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (r0, m0, g0, s0, t0), (r1, m1, g1, s1, t1) = out
    assert (r0, r1) == (0, 1)
    assert not set(m0) & set(m1) and sorted(m0 + m1) == list(range(10))
    assert (g0, g1) == (0, 1) and (s0, s1) == (0, 1)
    assert t0 == t1 == [20.0, 3.0]            # element-wise maximum on every rank
    assert R.throughput(100.0, world, 2.0) == 100.0


def test_single_process_needs_no_group():
    assert R.max_over_ranks(None, [1.5, 2.5], "cpu") == [1.5, 2.5]
    assert R.member_indices(3, 2) == [6, 7]
