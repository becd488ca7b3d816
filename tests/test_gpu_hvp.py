"""Orbital Hessian-vector product (las_orbital_hvp) against the oracle's analytic linearisation
of the gradient, in both precisions, on small ragged systems and the Nao=400 workload."""
import numpy as np
import pytest

from gpu_common import SMALL, built, dev, torch_cuda
from las_inputs import workload_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


def _X(s, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((s.nmo, s.nmo))
    return (X - X.T) / np.sqrt(2.0)


def _check(s, precision, tol, seed):
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    X = _X(s, seed)
    ref = O.orbital_hvp(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, X)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    dG, Dg = las.orbital_hvp(dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()), dev(X))
    las.sync()
    dG, Dg = dG.cpu().numpy(), Dg.cpu().numpy()
    las.close()
    assert np.abs(dG - ref["dG"]).max() <= tol * np.abs(ref["dG"]).max()
    assert np.abs(Dg - ref["Dg"]).max() <= tol * np.abs(ref["Dg"]).max()
    assert np.abs(Dg + Dg.T).max() == 0.0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("split", 1e-9)])
@pytest.mark.parametrize("name", ["nao48", "ragged", "nofrag", "nmo_lt_nao"])
def test_orbital_hvp_small(precision, tol, name):
    _check(SMALL[name](), precision, tol, seed=21)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("split", 1e-9),
                                           ("split_packed", 1e-9)])
def test_orbital_hvp_nao400(precision, tol):
    _check(workload_system("nao400"), precision, tol, seed=22)
