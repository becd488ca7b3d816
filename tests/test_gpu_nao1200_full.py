"""The whole Nao=1200 / Naux=4800 workload (27.7 GB of packed B), with the contexts the benchmark
times (default workspace, every auxiliary row in one context).

* The oracle evaluates the same system over all 4800 auxiliary functions (the full sums over P
  of Eqs. J_1-K_2 and ppaa; a few minutes on the host cores), and both precisions are compared
  with it element by element at the stated bars: FP64 |dE| <= 1e-10 |E| and max|d dE/dC| <= 1e-9;
  split |dE| <= 1e-8 Eh and max|d dE/dC| <= 1e-8, for both digit layouts of B (full rows, and
  the packed triangle with one exponent per auxiliary function).
* The energy and gradients are sums over L plus an h-linear term, so the whole-index context,
  whose B offsets pass 2^31 elements, must equal the sum of two contexts over the halves of the
  auxiliary index (each below 2^31 elements), the second one passed h = 0.  Both sides are split
  evaluations, each within the split bar of the exact value, so they may differ by twice it."""
import os
import time

import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import workload_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    torch = torch_cuda()
    built()
    torch.cuda.empty_cache()
    s = workload_system("nao1200")
    t0 = time.perf_counter()
    ref = O.system_energy_grad(s)
    t_oracle = time.perf_counter() - t0
    print(f"\noracle, whole Nao=1200 workload (4800 auxiliary rows, energy + dE/dC): "
          f"{t_oracle:.1f} s on {os.cpu_count()} host cores")
    B = dev(s.Bp)
    s.Bp = None   # the host copy (27.7 GB) is no longer needed
    yield s, B, ref
    del B
    torch.cuda.empty_cache()


def _eval(s, B, naux, precision, C, h, dm1s, dm2):
    from paper_2505_03755_gb300 import LasDF
    las = LasDF(B, s.nao, naux, s.nmo, s.ncore, s.nact, precision=precision)
    try:
        E, G = las.energy_grad(C, h, dm1s, dm2)
        las.sync()
        return float(E), G.cpu().numpy()
    finally:
        las.close()


@pytest.mark.parametrize("precision", ["fp64", "split", "split_packed"])
def test_nao1200_full_size_against_oracle(full, precision):
    s, B, ref = full
    assert B.numel() > 2**31
    E, G = _eval(s, B, s.naux, precision, dev(s.C), dev(s.h), dev(s.dm1s_flat()),
                 dev(s.dm2_flat()))
    dE = abs(E - ref["E"])
    dG = float(np.abs(G - ref["G"]).max())
    print(f"\n{precision}: E = {E:.10f}, |dE| = {dE:.3e} Eh, max|d dE/dC| = {dG:.3e} "
          f"(max|dE/dC| = {np.abs(ref['G']).max():.1f})")
    if precision == "fp64":
        assert dE <= 1e-10 * abs(ref["E"]), dE
        assert dG <= 1e-9, dG
    else:
        assert dE <= 1e-8, dE
        assert dG <= 1e-8, dG


def test_nao1200_whole_index_equals_its_halves(full):
    import torch
    s, B, _ = full
    C, h = dev(s.C), dev(s.h)
    dm1s, dm2 = dev(s.dm1s_flat()), dev(s.dm2_flat())
    Es, Gs = _eval(s, B, s.naux, "split", C, h, dm1s, dm2)
    half = s.naux // 2
    E0, G0 = _eval(s, B[:half], half, "split", C, h, dm1s, dm2)
    E1, G1 = _eval(s, B[half:], s.naux - half, "split", C, torch.zeros_like(h), dm1s, dm2)
    assert abs(E0 + E1 - Es) <= 2e-8, (E0 + E1, Es)
    assert np.abs(G0 + G1 - Gs).max() <= 2e-8
    # a half on its own is far from the whole (the partition is real)
    assert abs(E0 - Es) > 1e-3 * abs(Es)
