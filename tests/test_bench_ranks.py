"""The multi-rank bookkeeping of bench.py on two gloo ranks (CPU): each rank
runs its own replica (seed + rank), the reported time is the slowest rank's
and the attempts are summed over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, n = bench.combine_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, device="cpu")
    out.put((rank, ms, n, bench.replica_seed(1, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    assert [r[2] for r in res] == [3000, 3000]
    assert [r[3] for r in res] == [1, 2]


def test_single_rank_passthrough():
    import bench
    assert bench.combine_ranks(5.0, 7) == (5.0, 7)
