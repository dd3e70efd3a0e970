"""Host-side logic of the N-rank replica benchmark (gloo, world size 2, CPU only): the job step time
is the slowest rank's and the throughput counts every rank's units."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [4.0, 7.5][rank]
    value, t = bench.job_throughput(step_ms, 1_000_000, "cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_throughput():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, t = out[r]
        assert t == pytest.approx(7.5)
        assert value == pytest.approx(2 * 1_000_000 / 7.5e-3)


def test_single_process_is_identity():
    import bench
    value, t = bench.job_throughput(5.0, 1000, "cpu")
    assert t == 5.0 and value == pytest.approx(1000 / 5e-3)
