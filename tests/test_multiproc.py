"""Host-side logic of the N > 1 path (independent replicas, weak scaling) on
CPU ranks with the gloo backend: the job time is the max over ranks, every
rank draws its own noise, and the whole-job value counts all ranks' problems."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank            # rank 1 is the slow one
    ms = bench.job_time_ms(local_ms, world, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    dist.barrier()
    out[rank] = (ms, bench.job_value_s(ms, steps=4, world=world), tuple(seeds))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_max_and_count_all_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value, seeds = res[rank]
        assert ms == 125.0                       # max over ranks
        assert value == pytest.approx(0.125 / (4 * world))
        assert len(set(seeds)) == world          # independent noise per replica


def test_single_rank_needs_no_collective():
    assert bench.job_time_ms(42.0, 1) == 42.0
    assert bench.job_value_s(2000.0, 2, 1) == 1.0
