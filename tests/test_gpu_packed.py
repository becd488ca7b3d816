"""Split precision over the packed-triangle digit planes of B ("split_packed"): the lower 128 x 128
tiles of every b^L (diagonal tiles whole), each read as stored for its own row block and
transposed for its column block, plus the rows past the last whole 128-row block, with one power
of two per b^L.  Sizes cover no whole block (n < 128, every row ragged), whole blocks only
(n = 256), and whole blocks with ragged rows of one to 127; every result is compared with the
oracle at the split-mode bars, and with the full-row layout."""
import numpy as np
import pytest

from gpu_common import built, dev, gpu_energy_grad, make_las, torch_cuda
from las_inputs import batched_specs, make_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

E_ABS = 1e-8      # split mode: |dE| in Eh
G_ABS = 1e-8      # split mode: max-abs on dE/dC

SYSTEMS = {
    # (nao, naux, ncore, fragments (ne, m), seed): block structure of the packed layout
    "n100_ragged_only": (100, 130, 8, [(2, 3), (4, 4)], 31),
    "n256_whole_blocks": (256, 300, 20, [(4, 4), (2, 2)], 32),
    "n300_two_blocks_44": (300, 260, 24, [(3, 3), (4, 5), (2, 2)], 33),
    "n383_ragged_127": (383, 200, 30, [(4, 4)], 34),
    "n129_ragged_1": (129, 170, 10, [(2, 2), (2, 3)], 35),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_cuda()
    built()


def _system(name):
    n, X, c, frags, seed = SYSTEMS[name]
    return make_system(n, X, c, frags, seed=seed)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_packed_energy_grad_against_oracle(name):
    s = _system(name)
    ref = O.system_energy_grad(s)
    E, G, g = gpu_energy_grad(s, "split_packed")
    assert abs(E - ref["E"]) <= E_ABS, (E, ref["E"])
    assert np.abs(G - ref["G"]).max() <= G_ABS
    assert np.abs(g - ref["gorb"]).max() <= 10 * G_ABS
    # the full-row layout of the same system agrees within twice the bars
    E2, G2, _ = gpu_energy_grad(s, "split")
    assert abs(E - E2) <= 2 * E_ABS
    assert np.abs(G - G2).max() <= 2 * G_ABS


@pytest.mark.parametrize("name", ["n300_two_blocks_44", "n256_whole_blocks"])
def test_packed_df_jk_and_transform(name):
    """The JK call (the core density's half transform, Coulomb traces, exchange) and the AO2MO
    transform read B through the same packed products."""
    s = _system(name)
    las = make_las(s, "split_packed")
    J, K = las.df_jk(dev(s.C))
    a0, a1 = s.ncore, s.ncore + s.nactive
    lmu, lpu = las.df_transform(dev(s.C), 0, s.nmo)
    las.sync()
    ref = O.system_energy_grad(s, with_grad=False)
    assert np.abs(J.cpu().numpy() - ref["J"]).max() <= 1e-11 * np.abs(ref["J"]).max()
    assert np.abs(K.cpu().numpy() - ref["K"]).max() <= 1e-11 * np.abs(ref["K"]).max()
    rmu, rpu = O.df_transform(s.Bp, s.nao, s.C, (a0, a1), 0, s.nmo)
    assert np.abs(lmu.cpu().numpy() - rmu).max() <= 1e-11 * np.abs(rmu).max()
    assert np.abs(lpu.cpu().numpy() - rpu).max() <= 1e-11 * np.abs(rpu).max()
    las.close()


def test_packed_chunked_and_device_bytes():
    """Chunks of the auxiliary index start inside the tile array (a workspace cap that splits
    X into several chunks gives the same result), and the packed context holds fewer bytes."""
    s = _system("n300_two_blocks_44")
    E0, G0, _ = gpu_energy_grad(s, "split_packed")
    E1, G1, _ = gpu_energy_grad(s, "split_packed", max_workspace_bytes=8_000_000)
    assert abs(E1 - E0) <= 1e-10
    assert np.abs(G1 - G0).max() <= 1e-10
    a = make_las(s, "split")
    b = make_las(s, "split_packed")
    assert b.device_bytes() < a.device_bytes()
    a.close()
    b.close()


def test_packed_batched_matches_single_calls():
    """Packed contexts in the grouped batch: both products of each half transform (whole blocks
    and ragged rows) share the grouped launches; results are bit-identical to single calls."""
    torch = torch_cuda()
    from paper_2505_03755_gb300 import LasDF, energy_grad_batched
    specs = sorted(batched_specs(64), key=lambda x: x["nao"])
    chosen = [specs[0], specs[30], specs[45]]          # below, around and above 2 x 128 AOs
    systems = [make_system(x["nao"], x["naux"], x["ncore"], x["frags"], x["seed"]) for x in chosen]
    las, items = [], []
    for s in systems:
        L = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="split_packed")
        E = torch.empty((), dtype=torch.float64, device="cuda")
        G = torch.empty((s.nao, s.nmo), dtype=torch.float64, device="cuda")
        las.append(L)
        items.append((dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()), E, G))
    energy_grad_batched(las, items)
    torch.cuda.synchronize()
    for L, it, s in zip(las, items, systems):
        e0, g0 = float(it[4]), it[5].cpu().numpy()
        E, G = L.energy_grad(*it[:4])
        L.sync()
        assert float(E) == e0
        assert np.array_equal(G.cpu().numpy(), g0)
        if s.nao <= 300:
            ref = O.system_energy_grad(s)
            assert abs(e0 - ref["E"]) <= E_ABS
            assert np.abs(g0 - ref["G"]).max() <= G_ABS
    for L in las:
        L.close()
