"""Device-side failure detection without a GPU fault: a kernel waits on a barrier that nothing
signals; its bounded wait must give up, report LAS_ERR_TIMEOUT to the host and return, and the
device must stay usable for the next evaluation."""
import numpy as np
import pytest

from gpu_common import SMALL, built, gpu_energy_grad, torch_cuda
from oracle import las_oracle as O

pytestmark = pytest.mark.gpu

LAS_ERR_TIMEOUT = 4


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    torch = torch_cuda()
    built()
    from paper_2505_03755_gb300 import selftest_bounded_wait
    assert selftest_bounded_wait() == LAS_ERR_TIMEOUT
    torch.cuda.synchronize()
    # the context and the device keep working afterwards
    s = SMALL["nao48"]()
    ref = O.system_energy_grad(s)
    for precision in ("fp64", "split"):
        E, G, _ = gpu_energy_grad(s, precision, want_gorb=False)
        assert abs(E - ref["E"]) <= 1e-8
        assert np.abs(G - ref["G"]).max() <= 1e-8
    # and the self-test is repeatable
    assert selftest_bounded_wait() == LAS_ERR_TIMEOUT
