"""Effective potentials (Eqs. v_emb and vself) through las_veff, against the oracle, in both
precisions: the embedding potential of a LAS state with an open-shell fragment in the AO basis,
and the self potential of one fragment's own active density in an embedded basis."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import make_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


def _factored(C_c, C_a, g):
    """gamma = C_c C_c^T + C_a g C_a^T as (Cx, w) with g diagonalised."""
    lam, U = np.linalg.eigh(g)
    Cx = np.concatenate([C_c, C_a @ U], axis=1)
    w = np.concatenate([np.ones(C_c.shape[1]), lam])
    return np.ascontiguousarray(Cx), w, Cx @ np.diag(w) @ Cx.T


def _spin_blocks(dm1s, sigma):
    a = sum(d.shape[-1] for d in dm1s)
    g = np.zeros((a, a))
    off = 0
    for d in dm1s:
        m = d.shape[-1]
        g[off:off + m, off:off + m] = d[sigma]
        off += m
    return g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-11),
                                           ("split_packed", 1e-11)])
def test_veff_embedding_potential(precision, tol):
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(45, 90, 5, [(2, 2), (3, 3), (2, 3)], seed=4242)
    c, a = s.ncore, s.nactive
    fac = [_factored(s.C[:, :c], s.C[:, c:c + a], _spin_blocks(s.dm1s, sg)) for sg in range(2)]
    va_r, vb_r = O.embedding_potentials(s.Bp, s.nao, fac[0][2], fac[1][2])
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision=precision)
    va, vb = las.veff(dev(fac[0][0]), dev(fac[0][1]), dev(fac[1][0]), dev(fac[1][1]))
    las.sync()
    scale = max(np.abs(va_r).max(), np.abs(vb_r).max())
    assert np.abs(va.cpu().numpy() - va_r).max() <= tol * scale
    assert np.abs(vb.cpu().numpy() - vb_r).max() <= tol * scale
    las.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-11)])
def test_veff_self_potential_embedded_basis(precision, tol):
    """Eq. vself: the fragment's own active density in its embedded basis (no core part)."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    e = make_system(60, 120, 4, [(3, 4)], seed=4343)      # an embedded problem of 60 orbitals
    a0, ma = e.ncore, e.nactive
    M_a = e.C[:, a0:a0 + ma]
    empty = np.zeros((e.nao, 0))
    fac = [_factored(empty, M_a, e.dm1s[0][sg]) for sg in range(2)]
    va_r, vb_r = O.embedding_potentials(e.Bp, e.nao, fac[0][2], fac[1][2])
    las = LasDF(dev(e.Bp), e.nao, e.naux, e.nmo, e.ncore, e.nact, precision=precision)
    va, vb = las.veff(dev(fac[0][0]), dev(fac[0][1]), dev(fac[1][0]), dev(fac[1][1]))
    las.sync()
    scale = max(np.abs(va_r).max(), np.abs(vb_r).max())
    assert np.abs(va.cpu().numpy() - va_r).max() <= tol * scale
    assert np.abs(vb.cpu().numpy() - vb_r).max() <= tol * scale
    las.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-11)])
def test_veff_one_spin_empty(precision, tol):
    """gamma_beta = 0 (rank 0): v_alpha = J[gamma_a] - K[gamma_a], v_beta = J[gamma_a]."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(33, 50, 6, [], seed=4444)
    C_c = np.ascontiguousarray(s.C[:, :s.ncore])
    ga = C_c @ C_c.T
    va_r, vb_r = O.embedding_potentials(s.Bp, s.nao, ga, np.zeros_like(ga))
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, [], precision=precision)
    va, vb = las.veff(dev(C_c), dev(np.ones(s.ncore)), dev(np.zeros((s.nao, 0))),
                      dev(np.zeros(0)))
    las.sync()
    scale = max(np.abs(va_r).max(), np.abs(vb_r).max())
    assert np.abs(va.cpu().numpy() - va_r).max() <= tol * scale
    assert np.abs(vb.cpu().numpy() - vb_r).max() <= tol * scale
    las.close()
