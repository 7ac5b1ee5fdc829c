"""Multi-GPU path of bench.py ("replicas only"): each rank runs independent solves and the
job's time is the slowest rank's, its work the sum of all ranks'. Checked here with two
CPU processes on the gloo backend (no GPU)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, iters = bench.replica_totals(1.0 + rank, 100 * (rank + 1), "cpu")
    out[rank] = (secs, iters)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 300.0)


def test_single_process_is_identity():
    import bench
    assert bench.replica_totals(1.5, 7, "cpu") == (1.5, 7.0)
