"""L-partitioned evaluation on one GPU: contexts over blocks of auxiliary rows of B, evaluated
one after another in one process, whose shares add up to the whole system (the per-rank step of
the multi-GPU partition; the all-reduce itself is covered on CPU with gloo)."""
import functools

import numpy as np
import pytest

from gpu_common import SMALL, built, dev, gpu_energy_grad, torch_cuda
from las_inputs import workload_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_cuda()
    built()


def _sharded(s, precision, world):
    from paper_2505_03755_gb300 import LasDF, aux_range, aux_shard_partial
    C, h = dev(s.C), dev(s.h)
    dm1s, dm2 = dev(s.dm1s_flat()), dev(s.dm2_flat())
    total = None
    for r in range(world):
        l0, l1 = aux_range(s.naux, r, world)
        las = LasDF(dev(s.Bp[l0:l1]), s.nao, l1 - l0, s.nmo, s.ncore, s.nact,
                    precision=precision)
        buf, E, G, g = aux_shard_partial(las, C, h, dm1s, dm2, r, want_gorb=True)
        las.sync()
        parts = (float(E), G.cpu().numpy(), g.cpu().numpy())
        total = parts if total is None else tuple(a + b for a, b in zip(total, parts))
        las.close()
    return total


@pytest.mark.parametrize("precision,world", [("fp64", 2), ("fp64", 3), ("split", 3)])
@pytest.mark.parametrize("name", ["ragged", "nao48"])
def test_shards_add_up_small(name, precision, world):
    s = SMALL[name]()
    ref = O.system_energy_grad(s)
    E, G, g = _sharded(s, precision, world)
    E1, G1, g1 = gpu_energy_grad(s, precision)
    scale = max(1.0, np.abs(ref["G"]).max())
    # against the single context: FP64 mode differs only in the order of the sum over L; split
    # mode also in the digit exponents of the blocks (each within the split GEMM's bound)
    rel = 1e-12 if precision == "fp64" else 1e-10
    assert abs(E - E1) <= rel * max(1.0, abs(E1))
    assert np.abs(G - G1).max() <= rel * scale
    assert np.abs(g - g1).max() <= 10 * rel * scale
    # against the oracle with the bars of the unpartitioned parity tests
    tolE = 1e-10 * max(1.0, abs(ref["E"])) if precision == "fp64" else 1e-8
    tolG = 1e-9 if precision == "fp64" else 1e-8
    assert abs(E - ref["E"]) <= tolE
    assert np.abs(G - ref["G"]).max() <= tolG
    assert np.abs(g - ref["gorb"]).max() <= 10 * tolG


@functools.lru_cache(maxsize=None)
def _nao400():
    s = workload_system("nao400")
    return s, O.system_energy_grad(s)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_shards_add_up_nao400(precision):
    """Nao=400, Naux=1600 in three blocks (534, 533, 533 rows: ragged against every tile)."""
    s, ref = _nao400()
    E, G, g = _sharded(s, precision, 3)
    if precision == "fp64":
        assert abs(E - ref["E"]) <= 1e-10 * abs(ref["E"])
        assert np.abs(G - ref["G"]).max() <= 1e-9
    else:
        assert abs(E - ref["E"]) <= 1e-8
        assert np.abs(G - ref["G"]).max() <= 1e-8
    assert np.abs(g - ref["gorb"]).max() <= 1e-8
