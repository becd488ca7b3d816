"""Parity at the full Nao=1200 size of the benchmark workload: the oracle cannot evaluate all
4800 auxiliary functions in seconds, so both sides evaluate the same system (C, h, fragment RDMs
of the 1200-orbital workload) over two slices of its Cholesky vectors, the first and the last
120 auxiliary functions (rows of the same full-size seeded B), in both precisions."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import WORKLOADS, make_system, packed_B_rows
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

ROWS = 120


@pytest.fixture(scope="module")
def workload():
    c = WORKLOADS["nao1200"]
    s = make_system(c["nao"], c["naux"], c["ncore"], c["frags"], seed=c["seed"], with_B=False)
    slices = {}
    for l0 in (0, c["naux"] - ROWS):
        Bs = packed_B_rows(c["seed"], c["nao"], c["naux"], l0, l0 + ROWS)
        ref = O.energy_grad(Bs, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, with_grad=True)
        slices[l0] = (Bs, ref)
    return s, slices


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("which", ["first", "last"])
def test_nao1200_slice(workload, precision, which):
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, slices = workload
    l0 = min(slices) if which == "first" else max(slices)
    Bs, ref = slices[l0]
    las = LasDF(dev(Bs), s.nao, ROWS, s.nmo, s.ncore, s.nact, precision=precision)
    E, G = las.energy_grad(dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    las.sync()
    E, G = float(E), G.cpu().numpy()
    las.close()
    if precision == "fp64":
        assert abs(E - ref["E"]) <= 1e-10 * abs(ref["E"])
        assert np.abs(G - ref["G"]).max() <= 1e-11 * np.abs(ref["G"]).max()
    else:
        assert abs(E - ref["E"]) <= 1e-8          # Eh
        assert np.abs(G - ref["G"]).max() <= 1e-8
