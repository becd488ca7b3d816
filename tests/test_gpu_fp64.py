"""Parity of the native-FP64 GPU path against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest

from gpu_common import SMALL, built, dev, gpu_energy_grad, make_las, torch_cuda
from las_inputs import workload_system
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

E_REL = 1e-10     # FP64 mode: energy relative tolerance
G_ABS = 1e-9      # FP64 mode: max-abs tolerance on dE/dC


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_cuda()
    built()


@pytest.mark.parametrize("name", list(SMALL))
def test_energy_grad_small(name):
    s = SMALL[name]()
    ref = O.system_energy_grad(s)
    E, G, g = gpu_energy_grad(s, "fp64")
    assert abs(E - ref["E"]) <= E_REL * max(1.0, abs(ref["E"])), (E, ref["E"])
    assert np.abs(G - ref["G"]).max() <= G_ABS
    assert np.abs(g - ref["gorb"]).max() <= 10 * G_ABS


def test_energy_only_matches_grad_call():
    s = SMALL["ragged"]()
    las = make_las(s)
    E1 = las.energy(dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    E2, _ = las.energy_grad(dev(s.C), dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    las.sync()
    assert float(E1) == float(E2)
    las.close()


def test_chunked_workspace_same_result():
    s = SMALL["ragged"]()
    E0, G0, _ = gpu_energy_grad(s, "fp64")
    # a cap that forces several auxiliary chunks
    E1, G1, _ = gpu_energy_grad(s, "fp64", max_workspace_bytes=600_000)
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.abs(G1 - G0).max() <= 1e-12


def test_workspace_cap_too_small_is_reported():
    from paper_2505_03755_gb300 import LasError
    s = SMALL["nao48"]()
    with pytest.raises(LasError) as ei:
        make_las(s, max_workspace_bytes=1000)
    assert ei.value.code == 3  # LAS_ERR_WORKSPACE


def test_invalid_arguments():
    from paper_2505_03755_gb300 import LasDF, LasError
    s = SMALL["nao48"]()
    with pytest.raises(LasError) as ei:
        LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.nao, s.nact)   # ncore + a > nmo
    assert ei.value.code == 1
    with pytest.raises(LasError):
        LasDF(dev(s.Bp), s.nao, s.naux, s.nao + 1, s.ncore, s.nact)  # nmo > nao
    with pytest.raises(LasError):
        LasDF(dev(s.Bp), s.nao, s.naux, s.nmo, s.ncore, [2, 0])  # empty fragment


def test_wrong_shapes_are_rejected_before_launch():
    """Transposed or short buffers raise ValueError in the binding; the context still works."""
    torch = torch_cuda()
    s = SMALL["nmo_lt_nao"]()
    ref = O.system_energy_grad(s)
    las = make_las(s)
    C, h = dev(s.C), dev(s.h)
    dm1s, dm2 = dev(s.dm1s_flat()), dev(s.dm2_flat())
    with pytest.raises(ValueError):
        las.energy_grad(C.T.contiguous(), h, dm1s, dm2)                      # transposed C
    with pytest.raises(ValueError):
        las.energy_grad(C, h, dm1s, dm2, G=torch.empty((s.nao, s.nmo - 1), dtype=torch.float64,
                                                      device="cuda:0"))      # short output
    with pytest.raises(ValueError):
        las.energy_grad(C, h, dm1s, dm2[:-1])                                 # short 2-RDM
    with pytest.raises(ValueError):
        las.df_jk(C[:, :5].contiguous())
    with pytest.raises(ValueError):
        las.df_transform(C, 3, 2)
    E, G = las.energy_grad(C, h, dm1s, dm2)
    las.sync()
    assert abs(float(E) - ref["E"]) <= E_REL * max(1.0, abs(ref["E"]))
    assert np.abs(G.cpu().numpy() - ref["G"]).max() <= G_ABS
    las.close()


def test_host_entry_point_matches_device():
    s = SMALL["ragged"]()
    E0, G0, _ = gpu_energy_grad(s, "fp64")
    las = make_las(s)
    E1, G1 = las.energy_grad_host(np.ascontiguousarray(s.C), np.ascontiguousarray(s.h),
                                  s.dm1s_flat(), s.dm2_flat())
    las.close()
    assert E1 == E0
    assert np.array_equal(G1, G0)


def test_df_jk_matches_oracle():
    s = SMALL["ragged"]()
    las = make_las(s)
    J, K = las.df_jk(dev(s.C))
    las.sync()
    ref = O.system_energy_grad(s, with_grad=False)
    assert np.abs(J.cpu().numpy() - ref["J"]).max() <= 1e-11 * np.abs(ref["J"]).max()
    assert np.abs(K.cpu().numpy() - ref["K"]).max() <= 1e-11 * np.abs(ref["K"]).max()
    las.close()


def test_df_transform_matches_oracle():
    s = SMALL["ragged"]()
    las = make_las(s)
    a0, a1 = s.ncore, s.ncore + s.nactive
    lmu, lpu = las.df_transform(dev(s.C), 3, 30)
    las.sync()
    rmu, rpu = O.df_transform(s.Bp, s.nao, s.C, (a0, a1), 3, 30)
    assert np.abs(lmu.cpu().numpy() - rmu).max() <= 1e-12 * np.abs(rmu).max()
    assert np.abs(lpu.cpu().numpy() - rpu).max() <= 1e-12 * np.abs(rpu).max()
    las.close()


def test_autograd_backward_is_dEdC():
    torch = torch_cuda()
    from paper_2505_03755_gb300 import las_energy
    s = SMALL["nao48"]()
    las = make_las(s)
    C = dev(s.C).requires_grad_(True)
    E = las_energy(C, las, dev(s.h), dev(s.dm1s_flat()), dev(s.dm2_flat()))
    (3.0 * E).backward()
    ref = O.system_energy_grad(s)
    assert np.abs(C.grad.cpu().numpy() - 3.0 * ref["G"]).max() <= 3 * G_ABS
    las.close()


def test_nao400_energy_grad():
    s = workload_system("nao400")
    ref = O.system_energy_grad(s)
    E, G, g = gpu_energy_grad(s, "fp64")
    assert abs(E - ref["E"]) <= E_REL * abs(ref["E"])
    assert np.abs(G - ref["G"]).max() <= G_ABS
