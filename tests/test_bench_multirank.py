"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank gets its
own instances and the step time is the maximum over ranks."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    idx = bench.shard_indices(rank, world, 16)
    mx = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, idx)
    if rank == 0:
        out.put((gathered, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert mx == 20.0
    a, b = gathered
    assert len(a) == len(b) == 16 and not set(a) & set(b)
