"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each an independent replica, take the
max of their times and the sum of their work (replicas only: no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        red = bench.RankReducer(dist, "cpu")
        red.barrier()
        # rank r integrated 10 + r steps of a 1000-node replica in 2 + r seconds
        rate = bench.whole_job_rate(red, 1000, 10 + rank, 2.0 + rank)
        q.put((rank, rate, red.max(float(rank)), red.sum(1.0)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, mx, sm in out:
        # both ranks agree: (10 + 11) steps x 1000 nodes / max(2, 3) s
        assert rate == pytest.approx(21 * 1000 / 3.0)
        assert mx == 1.0 and sm == 2.0


def test_single_process_reducer_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    red = bench.RankReducer(None)
    assert red.max(3.5) == 3.5 and red.sum(2.0) == 2.0
    assert bench.whole_job_rate(red, 100, 4, 2.0) == 200.0
