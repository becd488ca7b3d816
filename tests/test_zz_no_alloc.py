"""The allocation-free GEMM entry point (for callers that cannot allocate device memory where
they need a product: host applications that own every device allocation through their own pool,
or loops where a cudaMalloc could synchronise the device).

It must give the same product as the allocating entry point, twice in a row (the shared scratch
array keeps the previous call's contents), and must refuse sizes beyond its fixed scratch.
This file is collected last so that a stop at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2505_03755_gb300 import load_library
    lib = load_library()
    L, vp = ctypes.c_long, ctypes.c_void_p
    lib.las_split_gemm_noalloc.argtypes = [L, L, L, vp, L, vp, L, vp, L, vp]
    lib.las_split_gemm_noalloc.restype = ctypes.c_int
    return torch, lib


def _noalloc(torch, lib, A, B):
    M, K = A.shape
    N = B.shape[1]
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.las_split_gemm_noalloc(M, N, K, A.data_ptr(), K, B.data_ptr(), N, C.data_ptr(), N,
                                    st)
    assert rc == 0, rc
    return C.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    torch, lib = _lib()
    from paper_2505_03755_gb300 import split_gemm
    rng = np.random.default_rng(11)
    for M, K, N in [(300, 1000, 200), (129, 257, 97)]:   # two calls in a row, new shapes
        A = torch.from_numpy(rng.standard_normal((M, K))).cuda()
        B = torch.from_numpy(rng.standard_normal((K, N))).cuda()
        ref = split_gemm(A, B).cpu().numpy()
        got = _noalloc(torch, lib, A, B)
        a, b = A.cpu().numpy(), B.cpu().numpy()
        rm = np.abs(a).max(axis=1)[:, None]
        cm = np.abs(b).max(axis=0)[None, :]
        assert np.all(np.abs(got - ref) <= 2.0 ** -43 * K * rm * cm)
        assert np.all(np.abs(got - a @ b) <= 2.0 ** -43 * K * rm * cm)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, lib = _lib()
    need = lib.las_split_gemm_workspace(4096, 4096, 4096)
    assert need > (64 << 20)
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.las_split_gemm_noalloc(4096, 4096, 4096, A.data_ptr(), 4096, A.data_ptr(), 4096,
                                    A.data_ptr(), 4096, None)
    assert rc == 3  # LAS_ERR_WORKSPACE, returned before any GPU work
