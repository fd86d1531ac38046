"""Multi-rank host logic with two CPU ranks (gloo): the perturbation shards partition the batch."""
import os
import socket

import pytest

from paper_2203_05623_gb300.shard import owned_perturbations


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_global, block, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = owned_perturbations(n_global, rank, world, block)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        q.put(got)


@pytest.mark.parametrize("n_global,block", [(64, 1), (64, 8), (37, 4)])
def test_shards_partition_the_batch_over_two_ranks(n_global, block):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_global, block, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(i for part in got for i in part)
    assert flat == list(range(n_global))
    assert all(got[r] == owned_perturbations(n_global, r, 2, block) for r in range(2))


def test_single_rank_owns_everything_and_bad_arguments_fail():
    assert owned_perturbations(10, 0, 1, 3) == list(range(10))
    with pytest.raises(ValueError):
        owned_perturbations(10, 2, 2)
