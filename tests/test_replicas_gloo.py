"""bench.py --gpus N runs N independent replicas (no data-path collective):
the cross-rank logic (timing barrier, max of the times, sum of the units) on
world_size-2 gloo process groups on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    d = bench.init_dist(w)
    d.barrier()
    t_max = bench.max_over_ranks(d, 10.0 + rank)          # per-rank times -> the slowest
    units = bench.sum_over_ranks(d, 1000 * (rank + 1))    # per-rank particle-steps -> the job's total
    out[rank] = (t_max, units)
    d.barrier()
    d.destroy_process_group()


def test_replica_timing_takes_max_time_and_total_units():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        assert out[rank] == (11.0, 3000.0)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.init_dist(1) is None
    assert bench.max_over_ranks(None, 5.0) == 5.0
    assert bench.sum_over_ranks(None, 7.0) == 7.0
