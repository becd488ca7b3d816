"""Fragment-embedding AO2MO (Eqs. ao2mo_1, ao2mo_2, ppaa, papa) through las_frag_ao2mo, against
the oracle on the same seeded inputs, in both precisions, on systems that span several GEMM
tiles with ragged edges, with the auxiliary index split into chunks and in one piece."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import make_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

CASES = [
    # (nao, naux, a0, ma, seed)
    (37, 53, 5, 3, 901),       # ragged everything
    (96, 200, 40, 8, 902),     # an embedded basis of 96 orbitals, 8 active
    (130, 150, 0, 6, 903),     # active block at the first columns, nmo*ma > one row tile
]


def _case(nao, naux, seed):
    s = make_system(nao, naux, 2, [(2, 2)], seed=seed)
    rng = np.random.default_rng(seed)
    # embedded MO coefficients: an orthogonal matrix plus a non-orthogonal perturbation
    M = s.C + 0.1 * rng.standard_normal(s.C.shape)
    return s, M


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-10),
                                           ("split_packed", 1e-10)])
@pytest.mark.parametrize("nao,naux,a0,ma,seed", CASES)
def test_frag_ao2mo(precision, tol, nao, naux, a0, ma, seed):
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, M = _case(nao, naux, seed)
    ppaa_r, papa_r = O.frag_ao2mo(s.Bp, s.nao, M, a0, ma)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    ppaa, papa = las.frag_ao2mo(dev(M), a0, ma)
    las.sync()
    assert np.abs(ppaa.cpu().numpy() - ppaa_r).max() <= tol * np.abs(ppaa_r).max()
    assert np.abs(papa.cpu().numpy() - papa_r).max() <= tol * np.abs(papa_r).max()
    # the second call reuses the workspace and gives the same numbers
    ppaa2, papa2 = las.frag_ao2mo(dev(M), a0, ma)
    las.sync()
    assert np.array_equal(ppaa2.cpu().numpy(), ppaa.cpu().numpy())
    assert np.array_equal(papa2.cpu().numpy(), papa.cpu().numpy())
    las.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-10)])
def test_frag_ao2mo_chunked(precision, tol):
    """A workspace cap small enough to split the auxiliary index into several chunks."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, M = _case(64, 300, 904)
    ppaa_r, papa_r = O.frag_ao2mo(s.Bp, s.nao, M, 10, 5)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision,
                max_workspace_bytes=16 << 20)
    ppaa, papa = las.frag_ao2mo(dev(M), 10, 5)
    las.sync()
    assert np.abs(ppaa.cpu().numpy() - ppaa_r).max() <= tol * np.abs(ppaa_r).max()
    assert np.abs(papa.cpu().numpy() - papa_r).max() <= tol * np.abs(papa_r).max()
    # only one of the outputs
    only_ppaa, none = las.frag_ao2mo(dev(M), 10, 5, want_papa=False)
    las.sync()
    assert none is None
    assert np.abs(only_ppaa.cpu().numpy() - ppaa_r).max() <= tol * np.abs(ppaa_r).max()
    las.close()


def test_frag_ao2mo_rejects_bad_ranges():
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, M = _case(20, 30, 905)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="fp64")
    for a0, ma in [(-1, 2), (19, 2), (0, 0)]:
        with pytest.raises(RuntimeError):
            las.frag_ao2mo(dev(M), a0, ma)
    las.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-10)])
@pytest.mark.parametrize("a0,ma", [(0, 24), (17, 7)])
def test_frag_ao2mo_active_range_edges(precision, tol, a0, ma):
    """Every orbital active (ma = nmo), and the active block ending at the last orbital."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, M = _case(24, 70, 906)
    ppaa_r, papa_r = O.frag_ao2mo(s.Bp, s.nao, M, a0, ma)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    ppaa, papa = las.frag_ao2mo(dev(M), a0, ma)
    las.sync()
    assert np.abs(ppaa.cpu().numpy() - ppaa_r).max() <= tol * np.abs(ppaa_r).max()
    assert np.abs(papa.cpu().numpy() - papa_r).max() <= tol * np.abs(papa_r).max()
    las.close()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_device_bytes_follow_workspace_growth(precision):
    """Growing the fragment workspace (ma 2 -> 4) leaves the context owning what a fresh context
    that only ran ma = 4 owns (freed buffers are no longer counted); a call that fits adds
    nothing; the transform's digit planes are counted once, on the first split-mode call."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s, M = _case(96, 200, 905)
    Md = dev(M)
    grown = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    fresh = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    b0 = grown.device_bytes()
    assert fresh.device_bytes() == b0
    grown.frag_ao2mo(Md, 10, 2)
    grown.frag_ao2mo(Md, 10, 4)
    fresh.frag_ao2mo(Md, 10, 4)
    grown.sync()
    fresh.sync()
    assert grown.device_bytes() == fresh.device_bytes() > b0
    grown.frag_ao2mo(Md, 10, 3)
    assert grown.device_bytes() == fresh.device_bytes()
    C = dev(s.C)
    b1 = grown.device_bytes()
    grown.df_transform(C, 0, s.nmo)
    b2 = grown.device_bytes()
    grown.df_transform(C, 0, s.nmo)
    grown.sync()
    assert grown.device_bytes() == b2
    assert (b2 > b1) == (precision == "split")
    grown.close()
    fresh.close()
