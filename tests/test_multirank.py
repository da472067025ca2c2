"""Host logic of the multi-GPU benchmark path, on CPU with gloo, world size 2:
each rank advances its own copy of the batch (independent simulations, no
data-path collective); the job's rate divides all ranks' node updates by the
slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max = bench.max_over_ranks(times[rank], "cpu")
    value = bench.weak_scaling_value(ms_max, nodes_per_step=1000, steps=10, world=world)
    out.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_uses_slowest_rank():
    world, times = 2, [200.0, 250.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 250.0
        # 2 ranks x 1000 nodes x 10 steps in 0.25 s
        assert value == pytest.approx(2 * 1000 * 10 / 0.25 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.weak_scaling_value(100.0, 500, 4, 1) == pytest.approx(500 * 4 / 0.1 / 1e6)
