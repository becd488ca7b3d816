"""Helpers for the GPU parity tests: device copies of the seeded inputs and the oracle runs."""
import functools

import numpy as np
import pytest

from las_inputs import workload_system, make_system


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@functools.lru_cache(maxsize=None)
def built():
    import __graft_entry__ as g
    g.build()
    return True


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


def make_las(s, precision="fp64", **kw):
    built()
    from paper_2505_03755_gb300 import LasDF
    return LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision, **kw)


def gpu_energy_grad(s, precision="fp64", want_gorb=True, **kw):
    las = make_las(s, precision, **kw)
    res = las.energy_grad(dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()),
                          want_gorb=want_gorb)
    E, G, g = res if want_gorb else (res[0], res[1], None)
    las.sync()
    out = float(E), G.cpu().numpy(), (g.cpu().numpy() if g is not None else None)
    las.close()
    return out


SMALL = {
    "nao48": lambda: workload_system("nao48"),
    # sizes that are multiples of no tile, three uneven fragments, one odd-electron fragment
    "ragged": lambda: make_system(37, 53, 5, [(2, 3), (3, 2), (4, 4)], seed=4242),
    "nofrag": lambda: make_system(29, 45, 6, [], seed=99),
    "onefrag_nocore": lambda: make_system(20, 33, 0, [(4, 4)], seed=7),
    "nmo_lt_nao": lambda: make_system(40, 70, 4, [(2, 2), (2, 3)], seed=8, nmo=30),
}
