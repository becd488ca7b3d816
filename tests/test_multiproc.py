"""Host-side multi-rank logic of the benchmark on CPU (gloo, world size 2): each rank owns an
independent problem (weak scaling, no data-path collective); the timed duration is the maximum
over ranks and the reported rate counts every rank's evaluations."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    # rank r "took" (r + 1) * 100 ms for 5 steps; the job time is the slowest rank's
    t = bench.max_over_ranks((rank + 1) * 0.1, ws)
    rate = bench.weak_scaling_rate(ws, 5, t)
    seeds = [None] * ws
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    out[rank] = (t, rate, tuple(seeds))
    dist.destroy_process_group()


def test_two_rank_timing_and_independent_problems():
    ws = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        t, rate, seeds = out[r]
        assert t == pytest.approx(0.2)          # max over ranks
        assert rate == pytest.approx(2 * 5 / 0.2)  # whole-job evaluations per second
        assert len(set(seeds)) == ws            # each rank draws its own system
