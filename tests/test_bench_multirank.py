"""The benchmark's multi-GPU path is replicas only: each rank factorizes its own matrix and the
ranks meet only to agree on the slowest rank's time.  This checks that aggregation with two
gloo ranks on the CPU (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    value, ms = bench.job_value(local_ms, steps=10, world=world, flops_per_step=1e9)
    bench.barrier(world)
    q.put((rank, value, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == pytest.approx(150.0)
        # both replicas' flops (2 x 10 x 1e9) over the slowest replica's 150 ms
        assert value == pytest.approx(2 * 10 * 1e9 / 0.150 / 1e9)


def test_single_rank_value():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_value(200.0, steps=4, world=1, flops_per_step=5e9)
    assert ms == 200.0 and value == pytest.approx(4 * 5e9 / 0.2 / 1e9)
