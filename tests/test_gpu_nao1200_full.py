"""The whole Nao=1200 / Naux=4800 workload (27.7 GB of packed B), with the contexts the benchmark
times (default workspace, every auxiliary row in one context).  The oracle cannot evaluate it
in seconds, so two properties that hold at any size stand in for it:

* the split path (BF16 digit products on tcgen05) and the native FP64 path (DMMA) are two
  independent GEMM engines over the same inputs, and must agree within the split bound;
* the energy and gradients are sums over L plus an h-linear term, so the whole-index context,
  whose B offsets pass 2^31 elements, must equal the sum of two contexts over the halves of the
  auxiliary index (each below 2^31 elements), the second one passed h = 0, within the split
  bound (the halves' digit exponents differ from the whole's).

The oracle itself pins the same system over its first and last auxiliary rows in
test_gpu_nao1200_slices.py."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import workload_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    torch = torch_cuda()
    built()
    torch.cuda.empty_cache()
    s = workload_system("nao1200")
    B = dev(s.Bp)
    s.Bp = None   # the host copy (27.7 GB) is no longer needed
    yield s, B
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


def test_nao1200_full_size(full):
    import torch
    s, B = full
    assert B.numel() > 2**31
    C, h = dev(s.C), dev(s.h)
    dm1s, dm2 = dev(s.dm1s_flat()), dev(s.dm2_flat())
    Es, Gs = _eval(s, B, s.naux, "split", C, h, dm1s, dm2)
    Ef, Gf = _eval(s, B, s.naux, "fp64", C, h, dm1s, dm2)
    gmax = np.abs(Gf).max()
    # split against native FP64: the energy bar in Eh; the gradient bar relative to max|dE/dC|
    # (the digit truncation error scales with the row and column maxima of each product)
    assert abs(Es - Ef) <= 1e-8, (Es, Ef)
    assert np.abs(Gs - Gf).max() <= 2e-11 * gmax, (np.abs(Gs - Gf).max(), gmax)
    # whole index against its two halves: the projection's digit exponents are taken over each
    # chunk of the auxiliary index, so the halves truncate differently; the split bound applies
    half = s.naux // 2
    E0, G0 = _eval(s, B[:half], half, "split", C, h, dm1s, dm2)
    E1, G1 = _eval(s, B[half:], s.naux - half, "split", C, torch.zeros_like(h), dm1s, dm2)
    assert abs(E0 + E1 - Es) <= 1e-8, (E0 + E1, Es)
    assert np.abs(G0 + G1 - Gs).max() <= 2e-11 * gmax
    # a half on its own is far from the whole (the partition is real)
    assert abs(E0 - Es) > 1e-3 * abs(Es)
