"""The multi-GPU path is replicas only: each rank steps its own lattice and
the job reports all ranks' lattice updates over the slowest rank's time.  Two
gloo ranks on the CPU exercise bench.py's cross-rank reduction."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [2.0, 3.0][rank]
    m = bench.max_over_ranks(local_seconds, "cpu", world)
    v = bench.aggregate_mlups(1_000_000, 100, m, world)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in out:
        assert m == 3.0
        assert v == pytest.approx(2 * 1_000_000 * 100 / 3.0 / 1e6)


def test_single_rank_is_plain_throughput():
    import bench
    assert bench.max_over_ranks(1.5, "cpu", 1) == 1.5
    assert bench.aggregate_mlups(4096, 1000, 2.0, 1) == pytest.approx(4096 * 1000 / 2.0 / 1e6)
