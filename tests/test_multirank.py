"""The multi-GPU path runs one independent replica per rank (the Hessian-action columns
and problems shard with no data-path collective); the only cross-rank step is the
max-over-ranks time used for the whole-job throughput.  Checked with two gloo ranks on
the CPU."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t_max = bench.weak_scaling_value(1.0 + rank, 600, world, "cpu")
    q.put((rank, value, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_value_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max in res:
        assert t_max == 2.0
        assert value == 2 * 600 / 2.0


def test_single_rank_value():
    import bench
    assert bench.weak_scaling_value(2.0, 120, 1) == (60.0, 2.0)
