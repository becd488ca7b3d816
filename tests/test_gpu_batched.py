"""Batched evaluation of uneven systems under one captured CUDA graph (split precision)."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import batched_specs, make_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_cuda()
    built()


def _systems(count, pick):
    specs = batched_specs(64)
    chosen = pick(specs)[:count]
    return [make_system(s["nao"], s["naux"], s["ncore"], s["frags"], s["seed"]) for s in chosen]


def _run(systems, cap=0):
    torch = torch_cuda()
    from paper_2505_03755_gb300 import LasDF, energy_grad_batched
    las, items = [], []
    for s in systems:
        Bd = dev(s.Bp)
        L = LasDF(Bd, s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="split",
                  max_workspace_bytes=cap)
        E = torch.empty((), dtype=torch.float64, device="cuda")
        G = torch.empty((s.nao, s.nmo), dtype=torch.float64, device="cuda")
        las.append(L)
        items.append((dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()), E, G))
    return las, items, energy_grad_batched


def test_batched_graph_matches_individual_and_oracle():
    torch = torch_cuda()
    # the smallest systems of the 64-system uneven workload (oracle-friendly) plus two larger
    systems = _systems(4, lambda sp: sorted(sp, key=lambda x: x["nao"])) + \
        _systems(2, lambda sp: sorted(sp, key=lambda x: -x["nao"])[20:])
    las, items, batched = _run(systems)
    las[0].autotune(*items[0][:4])
    # products of different tile widths in the same grouped launches
    las[1].set_tiles([64, 64, 64, 64])
    las[2].set_tiles([64, 96, 64, 96])
    batched(las, items)
    torch.cuda.synchronize()
    first = [(float(it[4]), it[5].cpu().numpy()) for it in items]
    # replay (same pointers) after perturbing nothing: identical results
    for it in items:
        it[4].zero_()
        it[5].zero_()
    batched(las, items)
    torch.cuda.synchronize()
    for (e0, g0), it in zip(first, items):
        assert float(it[4]) == e0
        assert np.array_equal(it[5].cpu().numpy(), g0)
    # each problem alone through the single-problem call gives the same numbers
    for L, it, (e0, g0) in zip(las, items, first):
        E, G = L.energy_grad(*it[:4])
        L.sync()
        assert float(E) == e0
        assert np.array_equal(G.cpu().numpy(), g0)
    # and the oracle agrees within the split-mode tolerances
    for s, (e0, g0) in list(zip(systems, first))[:4]:
        ref = O.system_energy_grad(s)
        assert abs(e0 - ref["E"]) <= 1e-8
        assert np.abs(g0 - ref["G"]).max() <= 1e-8
    for L in las:
        L.close()


def test_batched_graph_sees_new_inputs_on_replay():
    torch = torch_cuda()
    systems = _systems(3, lambda sp: sorted(sp, key=lambda x: x["nao"]))
    las, items, batched = _run(systems, cap=64 << 20)   # small cap: several chunks each
    batched(las, items)
    torch.cuda.synchronize()
    # new orbitals in the same buffers: the replayed graph must use them
    rng = np.random.default_rng(5)
    for s, it in zip(systems, items):
        import scipy.linalg as sl
        Xa = rng.standard_normal((s.nmo, s.nmo))
        U = sl.expm(0.01 * (Xa - Xa.T))
        s.C = np.ascontiguousarray(s.C @ U)
        it[0].copy_(dev(s.C))
    batched(las, items)
    torch.cuda.synchronize()
    for s, it in zip(systems, items):
        ref = O.system_energy_grad(s)
        assert abs(float(it[4]) - ref["E"]) <= 1e-8
        assert np.abs(it[5].cpu().numpy() - ref["G"]).max() <= 1e-8
    for L in las:
        L.close()


def test_batched_many_systems_share_branches():
    """More systems than graph branches (several per branch, shared out by size): every
    problem bit-identical to its single-problem call, the smallest against the oracle."""
    torch = torch_cuda()
    systems = _systems(13, lambda sp: sorted(sp, key=lambda x: x["nao"]))
    las, items, batched = _run(systems)
    batched(las, items)
    torch.cuda.synchronize()
    got = [(float(it[4]), it[5].cpu().numpy()) for it in items]
    for L, it, (e0, g0) in zip(las, items, got):
        E, G = L.energy_grad(*it[:4])
        L.sync()
        assert float(E) == e0
        assert np.array_equal(G.cpu().numpy(), g0)
    ref = O.system_energy_grad(systems[0])
    assert abs(got[0][0] - ref["E"]) <= 1e-8
    assert np.abs(got[0][1] - ref["G"]).max() <= 1e-8
    for L in las:
        L.close()


def test_batched_fp64_contexts_per_system_chains():
    """Native FP64 contexts are captured as whole per-system chains on the branches (no split
    products to group): bit-identical to single calls and at the FP64 bars against the oracle."""
    torch = torch_cuda()
    from paper_2505_03755_gb300 import LasDF, energy_grad_batched
    systems = _systems(3, lambda sp: sorted(sp, key=lambda x: x["nao"]))
    las, items = [], []
    for s in systems:
        las.append(LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="fp64"))
        items.append((dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()),
                      torch.empty((), dtype=torch.float64, device="cuda"),
                      torch.empty((s.nao, s.nmo), dtype=torch.float64, device="cuda")))
    energy_grad_batched(las, items)
    torch.cuda.synchronize()
    for s, L, it in zip(systems, las, items):
        e0, g0 = float(it[4]), it[5].cpu().numpy()
        E, G = L.energy_grad(*it[:4])
        L.sync()
        assert float(E) == e0 and np.array_equal(G.cpu().numpy(), g0)
        ref = O.system_energy_grad(s)
        assert abs(e0 - ref["E"]) <= 1e-10 * abs(ref["E"])
        assert np.abs(g0 - ref["G"]).max() <= 1e-9
        L.close()
