"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
ranks take disjoint seeded pairs and the step time is the max over ranks.
No GPU and no data-path collective are involved (pairs are independent)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synth import CONFIGS, make_pair
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    start = bench.shard_seed_offset(rank, 3)
    idx = list(range(start, start + 3))
    # a tiny pair per rank: distinct seeds give distinct data
    first = make_pair(CONFIGS["stress16x64"], idx[0])["src_range"].sum()
    t = torch.tensor([10.0 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    g = [None] * world
    dist.all_gather_object(g, (idx, float(first)))
    if rank == 0:
        out.put((float(t.item()), g))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_pairs_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    tmax, g = q.get()
    assert tmax == 20.0
    (i0, s0), (i1, s1) = g
    assert set(i0).isdisjoint(i1)
    assert s0 != s1
