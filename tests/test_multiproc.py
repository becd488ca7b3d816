"""Multi-rank logic on CPU (gloo, world size 2).

* The benchmark: each rank owns an independent problem (weak scaling, no data-path collective);
  the timed duration is the maximum over ranks and the reported rate counts every rank's
  evaluations.
* The L-partitioned evaluation: each rank holds a block of auxiliary rows of B, and one
  all-reduce of the ranks' shares gives the whole system's energy and gradients."""
import os
import socket

import numpy as np
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


# ------------------------------------------------------------------------------------------
# L-partitioned evaluation: each rank holds a block of auxiliary rows, one all-reduce (sum)
# ------------------------------------------------------------------------------------------
def test_aux_range_partitions_the_auxiliary_index():
    from paper_2505_03755_gb300 import aux_range
    for naux in (0, 1, 5, 53, 4800):
        for world in (1, 2, 3, 8):
            rs = [aux_range(naux, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == naux
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))      # contiguous, in rank order
            sizes = [l1 - l0 for l0, l1 in rs]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        aux_range(10, 2, 2)


class _OracleShard:
    """Stands in, on the CPU, for a context over auxiliary rows [l0, l1) of B: the oracle
    evaluates the energy and gradient from those rows only."""

    def __init__(self, s, l0, l1):
        self.s, self.l0, self.l1 = s, l0, l1

    def energy_grad(self, C, h, dm1s, dm2, want_gorb=False, E=None, G=None, g=None):
        from oracle import las_oracle as O
        s = self.s
        r = O.energy_grad(s.Bp, s.nao, h.numpy(), C.numpy(), s.ncore, s.dm1s, s.dm2,
                          l0=self.l0, l1=self.l1)
        E.fill_(r["E"])
        G.copy_(torch.from_numpy(r["G"]))
        if g is not None:
            g.copy_(torch.from_numpy(r["gorb"]))


def _shard_system():
    from las_inputs import make_system
    return make_system(17, 53, 3, [(2, 2), (3, 3)], seed=515)


def _sharded_worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2505_03755_gb300 import aux_range, energy_grad_aux_sharded
    s = _shard_system()
    l0, l1 = aux_range(s.naux, rank, ws)
    E, G, g = energy_grad_aux_sharded(_OracleShard(s, l0, l1), torch.from_numpy(s.C),
                                      torch.from_numpy(s.h), None, None, want_gorb=True)
    out[rank] = (float(E), G.numpy().copy(), g.numpy().copy(), (l0, l1))
    dist.destroy_process_group()


def test_two_rank_aux_sharded_energy_grad_equals_whole_system():
    """Rank 0 passes h, rank 1 a zero matrix; each evaluates its half of the auxiliary rows and
    one all-reduce gives every rank the whole system's E, dE/dC and rotation gradient."""
    from oracle import las_oracle as O
    ws = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_sharded_worker, args=(ws, port, out), nprocs=ws, join=True)
    s = _shard_system()
    ref = O.system_energy_grad(s)
    assert out[0][3] == (0, 27) and out[1][3] == (27, 53)
    for r in range(ws):
        E, G, g, _ = out[r]
        assert abs(E - ref["E"]) <= 1e-12 * abs(ref["E"])
        assert np.abs(G - ref["G"]).max() <= 1e-12 * np.abs(ref["G"]).max()
        assert np.abs(g - ref["gorb"]).max() <= 1e-12 * np.abs(ref["gorb"]).max()
    # a share on its own is not the answer (the partition is real)
    half = O.energy_grad(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, l0=0, l1=27)
    assert abs(half["E"] - ref["E"]) > 1e-6 * abs(ref["E"])



def _shard_worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w = dict(nao=11, naux=53, ncore=2, frags=[(2, 2), (2, 3)])
    s, (l0, l1), _ = bench.make_shard_inputs(rank, ws, w, seed=2024)
    t = bench.max_over_ranks(0.05 * (rank + 1), ws)
    out[rank] = (l0, l1, s.Bp.copy(), s.C.copy(), bench.strong_scaling_rate(4, t))
    dist.destroy_process_group()


def test_two_rank_partitioned_bench_inputs():
    """The bench's L-partition mode: each rank draws exactly its block of auxiliary rows of the
    same system (identical C on both ranks), the blocks tile the index, and the rate counts the
    one system's evaluations over the slowest rank's time."""
    from las_inputs import make_system
    ws = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_shard_worker, args=(ws, port, out), nprocs=ws, join=True)
    full = make_system(11, 53, 2, [(2, 2), (2, 3)], seed=2024)
    assert out[0][0] == 0 and out[0][1] == out[1][0] and out[1][1] == 53
    for r in range(ws):
        l0, l1, Bp, C, rate = out[r]
        assert np.array_equal(Bp, full.Bp[l0:l1])
        assert np.array_equal(C, full.C)
        assert rate == pytest.approx(4 / 0.1)
