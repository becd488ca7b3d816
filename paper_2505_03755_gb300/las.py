"""Thin Python binding of liblasdf (argument marshalling only; every step runs in CUDA).

PyTorch is used for device memory and streams.  All tensors passed in must be contiguous
float64 CUDA tensors.  Nothing here computes any part of the LAS energy or gradient: a missing
or unloadable shared library raises immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblasdf.so")

LAS_FP64 = 0
LAS_SPLIT_BF16 = 1
LAS_SPLIT_BF16_PACKED = 2
# "split_packed": split precision over packed-triangle digit planes of B (less memory)
PRECISIONS = {"fp64": LAS_FP64, "split": LAS_SPLIT_BF16, "split_bf16": LAS_SPLIT_BF16,
              "split_packed": LAS_SPLIT_BF16_PACKED}

EXPORTS = ["las_create", "las_destroy", "las_set_stream", "las_sync", "las_device_bytes",
           "las_df_transform", "las_df_jk", "las_energy", "las_energy_grad",
           "las_energy_grad_host", "las_set_timing", "las_stage_times", "las_kernel_launches",
           "las_split_gemm_workspace", "las_split_gemm", "las_energy_grad_batched",
           "las_autotune", "las_df_jk_density", "las_frag_ao2mo", "las_veff",
           "las_split_gemm_noalloc", "las_selftest_bounded_wait", "las_orbital_hvp",
           "las_probe_fp64", "las_get_tiles", "las_set_tiles", "las_status_str"]


class LasError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: status {code} ({msg})")
        self.code = code


class BatchItem(ctypes.Structure):
    _fields_ = [("C", ctypes.c_void_p), ("h", ctypes.c_void_p), ("dm1s", ctypes.c_void_p),
                ("dm2", ctypes.c_void_p), ("E", ctypes.c_void_p), ("dEdC", ctypes.c_void_p)]


class _Dims(ctypes.Structure):
    _fields_ = [("nao", ctypes.c_int), ("naux", ctypes.c_int), ("nmo", ctypes.c_int),
                ("ncore", ctypes.c_int), ("nfrag", ctypes.c_int),
                ("nact", ctypes.POINTER(ctypes.c_int))]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the in-tree liblasdf.so (built by paper_2505_03755_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblasdf.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.las_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Dims), vp, i, sz, vp]
    lib.las_destroy.argtypes = [vp]
    lib.las_set_stream.argtypes = [vp, vp]
    lib.las_sync.argtypes = [vp]
    lib.las_device_bytes.argtypes = [vp]
    lib.las_device_bytes.restype = sz
    lib.las_df_transform.argtypes = [vp, vp, i, i, vp, vp]
    lib.las_df_jk.argtypes = [vp, vp, vp, vp]
    lib.las_energy.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.las_energy_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.las_energy_grad_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.las_set_timing.argtypes = [vp, i]
    lib.las_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i]
    lib.las_stage_times.restype = i
    lib.las_split_gemm_workspace.argtypes = [ctypes.c_long] * 3
    lib.las_split_gemm_workspace.restype = sz
    lib.las_split_gemm.argtypes = [ctypes.c_long] * 3 + [vp, ctypes.c_long, vp, ctypes.c_long,
                                                         vp, ctypes.c_long, vp, sz, vp]
    lib.las_split_gemm.restype = i
    lib.las_energy_grad_batched.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(BatchItem), vp]
    lib.las_energy_grad_batched.restype = i
    lib.las_autotune.argtypes = [vp] * 7
    lib.las_autotune.restype = i
    lib.las_df_jk_density.argtypes = [vp, vp, vp, i, vp, vp]
    lib.las_df_jk_density.restype = i
    lib.las_frag_ao2mo.argtypes = [vp, vp, i, i, vp, vp]
    lib.las_frag_ao2mo.restype = i
    lib.las_veff.argtypes = [vp, vp, vp, i, vp, vp, i, vp, vp]
    lib.las_veff.restype = i
    lib.las_orbital_hvp.argtypes = [vp] * 8
    lib.las_orbital_hvp.restype = i
    lib.las_get_tiles.argtypes = [vp, ctypes.POINTER(i)]
    lib.las_get_tiles.restype = i
    lib.las_set_tiles.argtypes = [vp, ctypes.POINTER(i)]
    lib.las_set_tiles.restype = i
    lib.las_probe_fp64.argtypes = [ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), vp]
    lib.las_probe_fp64.restype = i
    lib.las_selftest_bounded_wait.argtypes = [vp]
    lib.las_selftest_bounded_wait.restype = i
    lib.las_kernel_launches.argtypes = []
    lib.las_kernel_launches.restype = ctypes.c_long
    lib.las_status_str.argtypes = [i]
    lib.las_status_str.restype = ctypes.c_char_p
    for name in ["las_create", "las_destroy", "las_set_stream", "las_sync", "las_df_transform",
                 "las_df_jk", "las_energy", "las_energy_grad", "las_energy_grad_host",
                 "las_set_timing"]:
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels liblasdf has launched in this process so far."""
    return int(load_library().las_kernel_launches())


def _check(code: int, where: str) -> None:
    if code != 0:
        msg = _lib.las_status_str(code).decode() if _lib is not None else "?"
        raise LasError(code, where, msg)


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("tensors must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _shape_check(t, shape, name: str) -> None:
    """Raise ValueError unless t (a tensor or array) has exactly `shape` (a tuple of ints) or,
    for a flat buffer, `shape` is an int and t holds that many elements.  The library cannot see
    the size of a device buffer, so this is what keeps a wrong argument from being read or
    written past its end."""
    got = tuple(t.shape)
    if isinstance(shape, int):
        n = int(np.prod(got)) if got else 1
        if n != shape:
            raise ValueError(f"{name}: expected {shape} elements, got shape {got}")
    elif got != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {got}")


def _hptr(a) -> int | None:
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("host buffers must be C-contiguous float64 numpy arrays")
    return a.ctypes.data


class LasDF:
    """One LAS problem (packed Cholesky vectors resident on the GPU) and its workspace."""

    def __init__(self, B_packed, nao: int, naux: int, nmo: int, ncore: int, nact: list[int],
                 precision: str = "fp64", max_workspace_bytes: int = 0, stream=None):
        import torch
        lib = load_library()
        self._lib = lib
        self.nao, self.naux, self.nmo, self.ncore = nao, naux, nmo, ncore
        self.nact = list(nact)
        self.precision = precision
        self._B = B_packed  # keep the referenced device buffer alive
        self._device = B_packed.device
        if B_packed.numel() != naux * nao * (nao + 1) // 2:
            raise ValueError("B_packed must hold naux * nao(nao+1)/2 values")
        arr = (ctypes.c_int * max(1, len(self.nact)))(*self.nact)
        self._nact_arr = arr
        dims = _Dims(nao, naux, nmo, ncore, len(self.nact), arr)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.las_create(ctypes.byref(h), ctypes.byref(dims), _ptr(B_packed),
                              PRECISIONS[precision], max_workspace_bytes,
                              self._stream.cuda_stream), "las_create")
        self._h = h

    @property
    def stream(self):
        return self._stream

    @property
    def nact_total(self) -> int:
        return sum(self.nact)

    def _arg(self, t, shape, name: str) -> int | None:
        """Device pointer of t after checking its shape and that it lives on the context's
        device (None passes through: the library checks which arguments are required)."""
        if t is None:
            return None
        _shape_check(t, shape, name)
        p = _ptr(t)
        if t.device != self._device:
            raise ValueError(f"{name}: on {t.device}, the context is on {self._device}")
        return p

    def _state_args(self, C, h, dm1s, dm2):
        n, nmo = self.nao, self.nmo
        return (self._arg(C, (n, nmo), "C"), self._arg(h, (n, n), "h"),
                self._arg(dm1s, sum(2 * m * m for m in self.nact), "dm1s"),
                self._arg(dm2, sum(m ** 4 for m in self.nact), "dm2"))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.las_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def release_packed_B(self) -> None:
        """Drop this object's reference to the packed Cholesky vectors.  A split-precision context
        keeps its own digit planes of B, so its energy, gradient, transform and fragment AO2MO
        calls never read B_packed again; the JK calls (df_jk, df_jk_density, veff) still do and
        raise after this call.  FP64 contexts read B_packed in every call and cannot release it."""
        if self.precision == "fp64":
            raise ValueError("an FP64 context reads B_packed in every call")
        self._B = None

    def _need_B(self, what: str) -> None:
        if self._B is None:
            raise ValueError(f"{what} reads B_packed, which this context has released")

    def device_bytes(self) -> int:
        return int(self._lib.las_device_bytes(self._h))

    def sync(self) -> None:
        _check(self._lib.las_sync(self._h), "las_sync")

    def set_timing(self, on: bool) -> None:
        _check(self._lib.las_set_timing(self._h, int(on)), "las_set_timing")

    def stage_times(self) -> list[float]:
        buf = (ctypes.c_float * 8)()
        k = self._lib.las_stage_times(self._h, buf, 8)
        return [buf[i] for i in range(k)]

    def energy(self, C, h, dm1s, dm2, E=None):
        import torch
        if E is None:
            E = torch.empty((), dtype=torch.float64, device=C.device)
        _check(self._lib.las_energy(self._h, *self._state_args(C, h, dm1s, dm2),
                                    self._arg(E, 1, "E")), "las_energy")
        return E

    def energy_grad(self, C, h, dm1s, dm2, want_gorb: bool = False, E=None, G=None, g=None):
        import torch
        dev = C.device
        if E is None:
            E = torch.empty((), dtype=torch.float64, device=dev)
        if G is None:
            G = torch.empty((self.nao, self.nmo), dtype=torch.float64, device=dev)
        if want_gorb and g is None:
            g = torch.empty((self.nmo, self.nmo), dtype=torch.float64, device=dev)
        _check(self._lib.las_energy_grad(self._h, *self._state_args(C, h, dm1s, dm2),
                                         self._arg(E, 1, "E"),
                                         self._arg(G, (self.nao, self.nmo), "G"),
                                         self._arg(g, (self.nmo, self.nmo), "g")),
               "las_energy_grad")
        return (E, G, g) if want_gorb else (E, G)

    def energy_grad_host(self, C, h, dm1s, dm2, with_grad: bool = True):
        E = np.zeros(1)
        G = np.empty((self.nao, self.nmo)) if with_grad else None
        n = self.nao
        for t, shape, name in ((C, (n, self.nmo), "C"), (h, (n, n), "h"),
                               (dm1s, sum(2 * m * m for m in self.nact), "dm1s"),
                               (dm2, sum(m ** 4 for m in self.nact), "dm2")):
            if t is not None:
                _shape_check(t, shape, name)
        _check(self._lib.las_energy_grad_host(self._h, _hptr(C), _hptr(h), _hptr(dm1s),
                                              _hptr(dm2), _hptr(E), _hptr(G)),
               "las_energy_grad_host")
        return float(E[0]), G

    def autotune(self, C, h, dm1s, dm2):
        """Pick, by timing, the fastest tile width of each split product kind and the fastest
        split-K factor of the projection GEMM for this problem."""
        import torch
        E = torch.empty((), dtype=torch.float64, device=C.device)
        G = torch.empty((self.nao, self.nmo), dtype=torch.float64, device=C.device)
        _check(self._lib.las_autotune(self._h, *self._state_args(C, h, dm1s, dm2), _ptr(E),
                                      _ptr(G)), "las_autotune")

    def tiles(self) -> list[int]:
        """Tile widths (64 or 96) of the split products: S1, S2, projection, one-electron."""
        buf = (ctypes.c_int * 4)()
        _check(self._lib.las_get_tiles(self._h, buf), "las_get_tiles")
        return list(buf)

    def set_tiles(self, widths) -> None:
        buf = (ctypes.c_int * 4)(*[int(w) for w in widths])
        _check(self._lib.las_set_tiles(self._h, buf), "las_set_tiles")

    def df_jk(self, C, J=None, K=None):
        import torch
        self._need_B("df_jk")
        n = self.nao
        J = torch.empty((n, n), dtype=torch.float64, device=C.device) if J is None else J
        K = torch.empty((n, n), dtype=torch.float64, device=C.device) if K is None else K
        _check(self._lib.las_df_jk(self._h, self._arg(C, (n, self.nmo), "C"),
                                   self._arg(J, (n, n), "J"), self._arg(K, (n, n), "K")),
               "las_df_jk")
        return J, K

    def df_jk_density(self, Cx, w, J=None, K=None):
        """J and K of D = Cx diag(w) Cx^T (Cx: n x r, w: r; device float64 tensors)."""
        import torch
        self._need_B("df_jk_density")
        n = self.nao
        J = torch.empty((n, n), dtype=torch.float64, device=Cx.device) if J is None else J
        K = torch.empty((n, n), dtype=torch.float64, device=Cx.device) if K is None else K
        if Cx.dim() != 2:
            raise ValueError("Cx must be nao x r")
        r = int(Cx.shape[1])
        _check(self._lib.las_df_jk_density(self._h, self._arg(Cx, (n, r), "Cx"),
                                           self._arg(w, (r,), "w"), r,
                                           self._arg(J, (n, n), "J"), self._arg(K, (n, n), "K")),
               "las_df_jk_density")
        return J, K

    def orbital_hvp(self, C, h, dm1s, dm2, X, want_Dg: bool = True):
        """(dG, Dg): the derivative of dE/dC along dC = C X and of the orbital-rotation gradient
        along C exp(tX), at fixed fragment RDMs (X antisymmetric nmo x nmo)."""
        import torch
        dev = C.device
        dG = torch.empty((self.nao, self.nmo), dtype=torch.float64, device=dev)
        Dg = torch.empty((self.nmo, self.nmo), dtype=torch.float64, device=dev) if want_Dg \
            else None
        _check(self._lib.las_orbital_hvp(self._h, *self._state_args(C, h, dm1s, dm2),
                                         self._arg(X, (self.nmo, self.nmo), "X"), _ptr(dG),
                                         _ptr(Dg)), "las_orbital_hvp")
        return dG, Dg

    def veff(self, C_alpha, w_alpha, C_beta, w_beta):
        """Effective potentials v_sigma = J[gamma_a + gamma_b] - K[gamma_sigma] (Eqs. v_emb,
        vself) of gamma_sigma = C_sigma diag(w_sigma) C_sigma^T (device float64 tensors)."""
        import torch
        self._need_B("veff")
        n, dev = self.nao, C_alpha.device
        va = torch.empty((n, n), dtype=torch.float64, device=dev)
        vb = torch.empty((n, n), dtype=torch.float64, device=dev)
        if C_alpha.dim() != 2 or C_beta.dim() != 2:
            raise ValueError("C_alpha and C_beta must be nao x r")
        ra, rb = int(C_alpha.shape[1]), int(C_beta.shape[1])
        _check(self._lib.las_veff(self._h, self._arg(C_alpha, (n, ra), "C_alpha"),
                                  self._arg(w_alpha, (ra,), "w_alpha"), ra,
                                  self._arg(C_beta, (n, rb), "C_beta"),
                                  self._arg(w_beta, (rb,), "w_beta"), rb, _ptr(va), _ptr(vb)),
               "las_veff")
        return va, vb

    def frag_ao2mo(self, M, a0: int, ma: int, want_ppaa: bool = True, want_papa: bool = True):
        """Fragment-embedding AO2MO (Eqs. ao2mo_1, ao2mo_2, ppaa, papa) in this context's basis:
        M (nao x nmo device float64) and the active columns [a0, a0+ma).  Returns (ppaa
        [nmo][nmo][ma][ma], papa [nmo][ma][nmo][ma]); either may be skipped."""
        import torch
        nmo, dev = self.nmo, M.device
        ppaa = torch.empty((nmo, nmo, ma, ma), dtype=torch.float64, device=dev) \
            if want_ppaa else None
        papa = torch.empty((nmo, ma, nmo, ma), dtype=torch.float64, device=dev) \
            if want_papa else None
        _check(self._lib.las_frag_ao2mo(self._h, self._arg(M, (self.nao, nmo), "M"), int(a0),
                                        int(ma), _ptr(ppaa), _ptr(papa)), "las_frag_ao2mo")
        return ppaa, papa

    def df_transform(self, C, p0: int, p1: int, want_lmu: bool = True, want_lpu: bool = True):
        import torch
        if not 0 <= p0 <= p1 <= self.nmo:
            raise ValueError("need 0 <= p0 <= p1 <= nmo")
        a = sum(self.nact)
        dev = C.device
        lmu = torch.empty((self.naux, self.nao, a), dtype=torch.float64, device=dev) \
            if want_lmu else None
        lpu = torch.empty((self.naux, p1 - p0, a), dtype=torch.float64, device=dev) \
            if want_lpu else None
        _check(self._lib.las_df_transform(self._h, self._arg(C, (self.nao, self.nmo), "C"), p0,
                                          p1, _ptr(lmu), _ptr(lpu)), "las_df_transform")
        return lmu, lpu


def selftest_bounded_wait(stream=None) -> int:
    """Run the device-side bounded-wait self-test; returns the las_status code it reports
    (LAS_ERR_TIMEOUT = 4 when the wait gave up as designed)."""
    import torch
    lib = load_library()
    st = (stream or torch.cuda.current_stream()).cuda_stream
    return int(lib.las_selftest_bounded_wait(st))


def probe_fp64(stream=None) -> tuple[float, float]:
    """Measured FP64 rates of the current device in TFLOP/s: (tensor-core MMA, fused
    multiply-add), from the library's register-resident probe loops."""
    import torch
    lib = load_library()
    st = (stream or torch.cuda.current_stream()).cuda_stream
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.las_probe_fp64(ctypes.byref(a), ctypes.byref(b), st), "las_probe_fp64")
    return a.value, b.value


def energy_grad_batched(problems, items, stream=None):
    """Evaluate many problems (LasDF objects) under one captured CUDA graph.

    items: list of (C, h, dm1s, dm2, E, dEdC) device tensors, one tuple per problem; the same
    tensors passed again replay the captured graph."""
    import torch
    lib = load_library()
    n = len(problems)
    arr = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
    if len(items) != n:
        raise ValueError("one item per problem")
    rows = []
    for p, (C, h, dm1s, dm2, E, G) in zip(problems, items):
        rows.append(BatchItem(*p._state_args(C, h, dm1s, dm2), p._arg(E, 1, "E"),
                              p._arg(G, (p.nao, p.nmo), "dEdC")))
    its = (BatchItem * n)(*rows)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib.las_energy_grad_batched(n, arr, its, st), "las_energy_grad_batched")


def aux_range(naux: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous block [l0, l1) of auxiliary indices that `rank` of `world` owns when the
    evaluation is partitioned along L (blocks differ in size by at most one row, in rank order)."""
    if world < 1 or not 0 <= rank < world or naux < 0:
        raise ValueError("need 0 <= rank < world and naux >= 0")
    q, r = divmod(naux, world)
    l0 = rank * q + min(rank, r)
    return l0, l0 + q + (1 if rank < r else 0)


def _aligned(k: int) -> int:
    return (k + 31) // 32 * 32


def aux_shard_partial(las, C, h, dm1s, dm2, rank: int, want_gorb: bool = False):
    """One rank's share of the energy and gradient when its context holds only its block of
    auxiliary rows of B (see `aux_range`).

    Every two-electron piece of the energy and of the gradient is a sum over L of per-L terms
    (v_L, T_L, Y_L, H_L; Eqs. J_1, K_1, ao2mo_1, ao2mo_2) and the one-electron matrix enters both
    linearly, so rank 0 alone passes h and the others a zero matrix: the ranks' shares then add
    up to the whole system's E, dE/dC and rotation gradient.  Returns (buf, E, G, g): the shares
    are views into the one flat device buffer `buf` (dE/dC, g, E at 256-byte-aligned offsets,
    zero padding between them), so a single sum over ranks of `buf` completes the evaluation."""
    import torch
    n, nmo = C.shape
    offg = _aligned(n * nmo)
    offE = offg + (_aligned(nmo * nmo) if want_gorb else 0)
    buf = torch.zeros(offE + 1, dtype=torch.float64, device=C.device)
    G = buf[:n * nmo].view(n, nmo)
    g = buf[offg:offg + nmo * nmo].view(nmo, nmo) if want_gorb else None
    E = buf[offE]
    hl = h if rank == 0 else torch.zeros_like(h)
    las.energy_grad(C, hl, dm1s, dm2, want_gorb=want_gorb, E=E, G=G, g=g)
    return buf, E, G, g


def energy_grad_aux_sharded(las, C, h, dm1s, dm2, want_gorb: bool = False, group=None):
    """E and dE/dC (and the rotation gradient) of the whole system, L-partitioned over the ranks
    of `group`: each rank evaluates its share (`aux_shard_partial`) and one all-reduce (sum) of
    the shares' flat buffer completes the evaluation on every rank.  Without an initialised
    process group (or with one rank) this is the plain single-context evaluation."""
    import torch.distributed as dist
    ws = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if ws > 1 else 0
    buf, E, G, g = aux_shard_partial(las, C, h, dm1s, dm2, rank, want_gorb)
    if ws > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return (E, G, g) if want_gorb else (E, G)


def split_gemm(A, B, out=None, stream=None):
    """C = A @ B (float64 CUDA tensors) through the emulated-FP64 BF16 tensor-core GEMM."""
    import torch
    lib = load_library()
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    C = torch.empty((M, N), dtype=torch.float64, device=A.device) if out is None else out
    _shape_check(C, (M, N), "out")
    # the library builds its tensor maps and launches on the current device
    cur = torch.device("cuda", torch.cuda.current_device())
    for t, name in ((A, "A"), (B, "B"), (C, "out")):
        if t.device != cur:
            raise ValueError(f"{name}: on {t.device}, the current CUDA device is {cur}")
    nbytes = int(lib.las_split_gemm_workspace(M, N, K))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib.las_split_gemm(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C),
                              C.stride(0), ws.data_ptr(), nbytes, st), "las_split_gemm")
    return C


def _energy_function():
    import torch

    class LasEnergy(torch.autograd.Function):
        """E(C) with the hand-written adjoint: forward runs las_energy_grad (when C needs a
        gradient) and keeps dE/dC; backward scales it by the incoming gradient."""

        @staticmethod
        def forward(ctx, C, las: LasDF, h, dm1s, dm2):
            if ctx.needs_input_grad[0]:
                E, G = las.energy_grad(C.detach().contiguous(), h, dm1s, dm2)
                ctx.save_for_backward(G)
            else:
                E = las.energy(C.detach().contiguous(), h, dm1s, dm2)
            return E

        @staticmethod
        def backward(ctx, gE):
            (G,) = ctx.saved_tensors
            return gE * G, None, None, None, None

    return LasEnergy


_LasEnergy = None


def las_energy(C, las: LasDF, h, dm1s, dm2):
    """Differentiable LAS energy E(C) (torch.autograd); dE/dC comes from the CUDA adjoint."""
    global _LasEnergy
    if _LasEnergy is None:
        _LasEnergy = _energy_function()
    return _LasEnergy.apply(C, las, h, dm1s, dm2)
