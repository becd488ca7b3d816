"""Split-precision (BF16 digit, tcgen05) path: the emulated-FP64 GEMM and the full LAS chain."""
import numpy as np
import pytest

from gpu_common import SMALL, built, dev, gpu_energy_grad, make_las, torch_cuda
from las_inputs import workload_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

E_ABS = 1e-8      # split mode: |dE| in Eh
G_ABS = 1e-8      # split mode: max-abs on dE/dC


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_cuda()
    built()


def _gemm(A, B):
    from paper_2505_03755_gb300 import split_gemm
    C = split_gemm(dev(A), dev(B))
    return C.cpu().numpy()


def test_split_gemm_integer_inputs_bit_exact():
    rng = np.random.default_rng(1)
    A = rng.integers(-100, 101, size=(300, 1000)).astype(np.float64)
    B = rng.integers(-100, 101, size=(1000, 200)).astype(np.float64)
    C = _gemm(A, B)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(C, ref)


def _digit_matrix(rows, cols, which, rng):
    """Entries sum_s d_s 2^(-7-8s) over the digit positions `which` (|d_s| < 128); the first
    column is 0.75 so that every row maximum lies in [0.5, 1)."""
    a = np.zeros((rows, cols))
    for s in which:
        a += rng.integers(-127, 128, size=(rows, cols)).astype(np.float64) * 2.0 ** (-7 - 8 * s)
    a[:, 0] = 0.75
    return a


@pytest.mark.parametrize("wa,wb", [([0], [0]), ([1], [0]), ([0], [1]), ([1], [1]), ([2], [0]),
                                   ([0, 1], [0, 1]), ([3], [0]), ([0], [3]), ([1], [2]),
                                   ([0, 1, 2], [0, 1]), ([4], [0])])
def test_split_gemm_digit_groups_bit_exact(wa, wb):
    """Operands made of chosen BF16 digits: every kept digit product is formed exactly (the four
    leading weight groups accumulate exactly; a single tail weight is exact in FP32), so the
    result equals the exact product bit for bit.  (Weight 2^-40 alone is not tested this way: an
    exact result with terms 2^-54 below its leading term is not representable in FP64.)"""
    rng = np.random.default_rng(len(wa) * 10 + sum(wa) + 7 * sum(wb))
    A = _digit_matrix(128, 352, wa, rng)
    B = np.ascontiguousarray(_digit_matrix(96, 352, wb, rng).T)
    assert np.array_equal(_gemm(A, B), A @ B)


def test_split_gemm_large_exact_sums_bit_exact():
    """Digit products of one sign: the exact-group partial sums of a 256-long chunk come close to
    their 2^24 bound (group 1: 2 * 127 * 72 * 256 = 4.7e6 in units of 2^-8), next to rows of
    mixed-sign digits (rows 64..127) in the same tiles.  Every entry has two digits, so the
    product is exact in FP64 and the split result must equal it bit for bit."""
    rng = np.random.default_rng(11)
    a = 127 * 2.0 ** -7 - 72 * 2.0 ** -15          # digits d_0 = 127, d_1 = -72
    A = np.full((256, 1024), a)
    A[64:128] = _digit_matrix(64, 1024, [0, 1], rng)
    A[192:] = -a
    B = np.full((1024, 160), a)
    B[:, 100:] = _digit_matrix(60, 1024, [0, 1], rng).T
    C = _gemm(A, B)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("M,K,N", [(1, 5, 3), (128, 32, 96), (257, 1111, 190), (130, 700, 16)])
def test_split_gemm_random_fp64(M, K, N):
    rng = np.random.default_rng(M + K + N)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, size=(1, N)))
    C = _gemm(A, B)
    ref = A @ B
    # error budget per product term, relative to row max x column max: operand rounding
    # (2 x 2^-48), dropped digit pairs of weight 2^-48 (5 x 2^-48) and the FP32 tail of weights
    # 2^-32 and 2^-40 (11 x 2^-56), i.e. below 2^-43 * K * rowmax * colmax
    rm = np.abs(A).max(axis=1)[:, None]
    cm = np.abs(B).max(axis=0)[None, :]
    err = np.abs(C - ref)
    assert np.all(err <= 2.0 ** -43 * K * rm * cm), (err / (K * rm * cm)).max()
    # and the typical error (random signs) grows like sqrt(K), well below the worst case
    assert np.sqrt(np.mean((err / (rm * cm)) ** 2)) <= 2.0 ** -44 * np.sqrt(K)


@pytest.mark.parametrize("name", list(SMALL))
def test_energy_grad_small_split(name):
    s = SMALL[name]()
    ref = O.system_energy_grad(s)
    E, G, g = gpu_energy_grad(s, "split")
    assert abs(E - ref["E"]) <= E_ABS, (E, ref["E"])
    assert np.abs(G - ref["G"]).max() <= G_ABS
    assert np.abs(g - ref["gorb"]).max() <= 10 * G_ABS


def test_split_chunked_workspace_same_result():
    s = SMALL["ragged"]()
    E0, G0, _ = gpu_energy_grad(s, "split")
    E1, G1, _ = gpu_energy_grad(s, "split", max_workspace_bytes=2_000_000)
    assert abs(E1 - E0) <= 1e-10
    assert np.abs(G1 - G0).max() <= 1e-10


def test_split_autograd():
    from paper_2505_03755_gb300 import las_energy
    s = SMALL["nao48"]()
    las = make_las(s, "split")
    C = dev(s.C).requires_grad_(True)
    E = las_energy(C, las, dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    E.backward()
    ref = O.system_energy_grad(s)
    assert np.abs(C.grad.cpu().numpy() - ref["G"]).max() <= G_ABS
    las.close()


def test_nao400_split():
    s = workload_system("nao400")
    ref = O.system_energy_grad(s)
    E, G, _ = gpu_energy_grad(s, "split", want_gorb=False)
    assert abs(E - ref["E"]) <= E_ABS
    assert np.abs(G - ref["G"]).max() <= G_ABS


@pytest.mark.parametrize("name", ["ragged", "nao48"])
def test_split_df_jk(name):
    s = SMALL[name]()
    las = make_las(s, "split")
    J, K = las.df_jk(dev(s.C))
    las.sync()
    ref = O.system_energy_grad(s, with_grad=False)
    assert np.abs(J.cpu().numpy() - ref["J"]).max() <= 1e-11 * np.abs(ref["J"]).max()
    assert np.abs(K.cpu().numpy() - ref["K"]).max() <= 1e-11 * np.abs(ref["K"]).max()
    las.close()


@pytest.mark.parametrize("name,p0,p1", [("ragged", 3, 30), ("nao48", 0, 48), ("nmo_lt_nao", 5, 30)])
def test_split_df_transform(name, p0, p1):
    """(L|mu u) and (L|pu) (Eqs. ao2mo_1, ao2mo_2) in split precision, p over a ragged range."""
    s = SMALL[name]()
    las = make_las(s, "split")
    a0, a1 = s.ncore, s.ncore + s.nactive
    lmu, lpu = las.df_transform(dev(s.C), p0, p1)
    las.sync()
    rmu, rpu = O.df_transform(s.Bp, s.nao, s.C, (a0, a1), p0, p1)
    assert np.abs(lmu.cpu().numpy() - rmu).max() <= 1e-11 * np.abs(rmu).max()
    assert np.abs(lpu.cpu().numpy() - rpu).max() <= 1e-11 * np.abs(rpu).max()
    las.close()


def test_split_df_transform_chunked_nao400():
    """The Nao=400 workload with a workspace cap that splits the auxiliary index into chunks."""
    s = workload_system("nao400")
    las = make_las(s, "split", max_workspace_bytes=256 << 20)
    a0, a1 = s.ncore, s.ncore + s.nactive
    lmu, lpu = las.df_transform(dev(s.C), 0, s.nmo)
    las.sync()
    rmu, rpu = O.df_transform(s.Bp, s.nao, s.C, (a0, a1), 0, s.nmo)
    assert np.abs(lmu.cpu().numpy() - rmu).max() <= 1e-11 * np.abs(rmu).max()
    assert np.abs(lpu.cpu().numpy() - rpu).max() <= 1e-11 * np.abs(rpu).max()
    las.close()


def test_split_context_releases_packed_B():
    """A split context keeps its own digit planes of B: after release_packed_B (and the buffer
    freed) the energy and gradient are unchanged, and the JK calls, which read B_packed,
    refuse instead of reading freed memory."""
    torch = torch_cuda()
    from gpu_common import SMALL
    from paper_2505_03755_gb300 import LasDF
    s = SMALL["ragged"]()
    B = dev(s.Bp)
    las = LasDF(B, s.nao, s.naux, s.nmo, s.ncore, s.nact, precision="split")
    args = (dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    E0, G0 = las.energy_grad(*args)
    las.sync()
    e0, g0 = float(E0), G0.cpu().numpy()
    las.release_packed_B()
    del B
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    E1, G1 = las.energy_grad(*args)
    las.sync()
    assert float(E1) == e0 and np.array_equal(G1.cpu().numpy(), g0)
    with pytest.raises(ValueError):
        las.df_jk(args[0])
    las.close()


def test_tile_widths_give_identical_results():
    """The tile width (64 or 96 output columns) only regroups output columns: every element sums
    the same digit products in the same order, so the results are bit-identical.  Nao=400
    (76 occupied orbitals: one 96-column tile or two 64-column tiles)."""
    torch_cuda()
    s = workload_system("nao400")
    las = make_las(s, "split")
    args = (dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    out = {}
    for widths in ([96, 96, 96, 96], [64, 64, 64, 64], [64, 96, 64, 96]):
        las.set_tiles(widths)
        assert las.tiles() == widths
        E, G = las.energy_grad(*args)
        las.sync()
        out[tuple(widths)] = (float(E), G.cpu().numpy())
    e0, g0 = out[(96, 96, 96, 96)]
    for e, g in out.values():
        assert e == e0 and np.array_equal(g, g0)
    with pytest.raises(Exception):
        las.set_tiles([80, 96, 96, 96])
    las.close()
