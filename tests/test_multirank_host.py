"""Host side of the multi-process benchmark path (`--gpus N` runs N
independent replicas, one per rank): the cross-rank reductions and the
whole-job throughput, on two CPU ranks over gloo."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws2, rank2, local = bench._dist()
        bench._barrier(ws)
        # rank r did (r + 1) * 1000 units in (r + 2) seconds
        units, secs = (rank + 1) * 1000.0, rank + 2.0
        q.put((rank, ws2, rank2, local, bench._sum_over_ranks(units, ws), bench._max_over_ranks(secs, ws),
               bench.replica_value(units, secs, ws)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_reductions():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, rank2, local, tot, slow, value in out:
        assert (ws, rank2, local) == (2, rank, rank)
        assert tot == 3000.0 and slow == 3.0
        assert value == pytest.approx(1000.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._sum_over_ranks(5.0, 1) == 5.0 and bench._max_over_ranks(2.0, 1) == 2.0
    assert bench.replica_value(10.0, 4.0, 1) == 2.5
