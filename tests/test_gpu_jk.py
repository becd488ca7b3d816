"""The general-density JK call (Eqs. J_1-K_2) through las_df_jk_density, against the oracle's
JK of the explicit density D = Cx diag(w) Cx^T (mixed-sign weights), in both precisions."""
import numpy as np
import pytest

from gpu_common import built, dev, torch_cuda
from las_inputs import make_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-11),
                                           ("split_packed", 1e-11)])
@pytest.mark.parametrize("r", [1, 12, 30])
def test_df_jk_density(precision, tol, r):
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(37, 53, 30, [], seed=606)      # a JK context: ncore >= r, no fragments
    rng = np.random.default_rng(r)
    Cx = rng.standard_normal((s.nao, r))
    w = rng.standard_normal(r)
    D = Cx @ np.diag(w) @ Cx.T
    (Jr,), (Kr,) = O.df_jk(s.Bp, s.nao, [D])
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, [], precision=precision)
    J, K = las.df_jk_density(dev(Cx), dev(w))
    las.sync()
    assert np.abs(J.cpu().numpy() - Jr).max() <= tol * np.abs(Jr).max()
    assert np.abs(K.cpu().numpy() - Kr).max() <= tol * np.abs(Kr).max()
    las.close()


def test_df_jk_density_spin_densities_of_a_las_state():
    """gamma_sigma = C_c C_c^T + C_a gamma^act_sigma C_a^T: the per-spin K of Eq. v_emb,
    with the active block diagonalised on the host to give the factored form."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(40, 70, 4, [(2, 2), (3, 3)], seed=77)
    Dact, _ = O.active_rdms(s.dm1s, s.dm2)
    c, a = s.ncore, s.nactive
    for sigma in range(2):
        g = np.zeros((a, a))
        off = 0
        for d in s.dm1s:
            m = d.shape[-1]
            g[off:off + m, off:off + m] = d[sigma]
            off += m
        lam, U = np.linalg.eigh(g)
        Cx = np.concatenate([s.C[:, :c], s.C[:, c:c + a] @ U], axis=1)
        w = np.concatenate([np.ones(c), lam])
        D = s.C[:, :c] @ s.C[:, :c].T + s.C[:, c:c + a] @ g @ s.C[:, c:c + a].T
        (Jr,), (Kr,) = O.df_jk(s.Bp, s.nao, [D])
        las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="split")
        J, K = las.df_jk_density(dev(Cx), dev(w))
        las.sync()
        assert np.abs(J.cpu().numpy() - Jr).max() <= 1e-11 * np.abs(Jr).max()
        assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-11 * np.abs(Kr).max()
        las.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-11)])
def test_df_jk_density_weight_edge_cases(precision, tol):
    """All weights negative, zero weights mixed in, and the empty density (r = 0)."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(41, 60, 20, [], seed=6060)
    rng = np.random.default_rng(3)
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, [], precision=precision)
    Cx = rng.standard_normal((s.nao, 9))
    for w in (-np.abs(rng.standard_normal(9)),
              np.where(np.arange(9) % 3 == 0, 0.0, rng.standard_normal(9))):
        D = Cx @ np.diag(w) @ Cx.T
        (Jr,), (Kr,) = O.df_jk(s.Bp, s.nao, [D])
        J, K = las.df_jk_density(dev(Cx), dev(w))
        las.sync()
        assert np.abs(J.cpu().numpy() - Jr).max() <= tol * np.abs(Jr).max()
        assert np.abs(K.cpu().numpy() - Kr).max() <= tol * np.abs(Kr).max()
    J, K = las.df_jk_density(dev(np.zeros((s.nao, 0))), dev(np.zeros(0)))
    las.sync()
    assert not J.abs().max().item() and not K.abs().max().item()
    las.close()


@pytest.mark.parametrize("precision", ["split", "split_packed"])
@pytest.mark.parametrize("r", [100, 150, 170])
def test_split_df_jk_density_two_tile_widths(r, precision):
    """Density ranks past one 96-column tile: r = 100 and 150 run the half transform as a
    96-column product plus a 64-column product over the remaining columns (4 and 54 of them);
    r = 170 leaves 74 and stays in 96-column tiles.  All against the oracle's JK, for both digit
    layouts of B (180 AOs: one whole 128-row block and 52 ragged rows when packed)."""
    torch_cuda()
    built()
    from paper_2505_03755_gb300 import LasDF
    s = make_system(180, 64, 170, [], seed=1505)
    rng = np.random.default_rng(r + 1)
    Cx = rng.standard_normal((s.nao, r))
    w = rng.standard_normal(r)
    D = Cx @ np.diag(w) @ Cx.T
    (Jr,), (Kr,) = O.df_jk(s.Bp, s.nao, [D])
    las = LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, [], precision=precision)
    J, K = las.df_jk_density(dev(Cx), dev(w))
    las.sync()
    assert np.abs(J.cpu().numpy() - Jr).max() <= 1e-11 * np.abs(Jr).max()
    assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-11 * np.abs(Kr).max()
    las.close()
