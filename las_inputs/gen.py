"""Seeded synthetic inputs for density-fitted LAS energy/gradient evaluations.

This module only *draws* inputs; it contains none of the LAS/DF arithmetic. Both the CPU
oracle (tests) and the GPU library (tests, bench) receive the arrays produced here.

Random numbers come from a counter-based generator so that any element of a large tensor
can be drawn independently (and in parallel chunks) from (seed, stream, index):

* ``splitmix64`` is the published 64-bit finaliser of Steele, Lea and Flood ("Fast
  splittable pseudorandom number generators", OOPSLA 2014), constants as published.
* element ``i`` of stream ``s`` is ``splitmix64(key_s + i)`` with
  ``key_s = splitmix64(seed * 2**32 + s)``;
* a uniform in (0,1) is ``((v >> 11) + 0.5) * 2**-53``;
* a standard normal is one Box-Muller draw, ``sqrt(-2 ln u1) cos(2 pi u2)``, from the two
  uniforms at counters ``2i`` and ``2i+1``.

Shapes and value distributions follow the workloads of the paper (Section "Identification of
computational bottlenecks", Eq. cholesky; the packed lower-triangular storage of the Cholesky
vectors described under "Calculation of effective potentials"):

* ``B[L, mu*(mu+1)/2 + nu] = N(0,1) * exp(-|mu-nu|/8) * exp(-L/Naux)`` for mu >= nu (stream 0);
* ``h`` symmetric, lower triangle ``N(0,1) * exp(-|mu-nu|/8)`` (stream 1), mirrored;
* ``C`` the Q factor of a Householder QR of an n x n Gaussian (stream 2), column signs fixed
  so that diag(R) > 0;
* one CI vector per fragment (stream 3 + K), Gaussian over alpha-string x beta-string, Ms = 0,
  normalised.  Fragment RDMs follow from it (``las_inputs.rdm``).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 20250503


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 finaliser on uint64 (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GAMMA)
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    v = (int(seed) * (1 << 32) + int(stream)) & 0xFFFFFFFFFFFFFFFF
    return splitmix64(np.array([v], dtype=np.uint64))[0]


def uniforms(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(start, start + count, dtype=np.uint64) + key
    v = splitmix64(ctr)
    return ((v >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normals(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normals with element indices [start, start+count) of a stream."""
    u = uniforms(seed, stream, 2 * start, 2 * count)
    u1 = u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def npair(n: int) -> int:
    return n * (n + 1) // 2


def _tril_decay(n: int) -> np.ndarray:
    """exp(-|mu-nu|/8) in packed lower-triangular order mu(mu+1)/2 + nu."""
    mu, nu = np.tril_indices(n)
    return np.exp(-np.abs(mu - nu).astype(np.float64) / 8.0)


def packed_B(seed: int, n: int, naux: int, out: np.ndarray | None = None,
             threads: int | None = None) -> np.ndarray:
    """B[L, p] for L in [0, naux), p the packed (mu >= nu) pair index; float64, C order."""
    P = npair(n)
    if out is None:
        out = np.empty((naux, P), dtype=np.float64)
    decay = _tril_decay(n)

    def rows(l0: int, l1: int) -> None:
        for L in range(l0, l1):
            z = normals(seed, 0, L * P, P)
            z *= decay
            z *= np.exp(-L / naux)
            out[L] = z

    threads = threads or min(32, os.cpu_count() or 1)
    step = max(1, (naux + threads * 4 - 1) // (threads * 4))
    if naux * P < 4_000_000 or threads == 1:
        rows(0, naux)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda a: rows(a, min(naux, a + step)), range(0, naux, step)))
    return out


def packed_B_rows(seed: int, n: int, naux: int, l0: int, l1: int,
                  threads: int | None = None) -> np.ndarray:
    """Rows [l0, l1) of the full-size packed B of `packed_B(seed, n, naux)` (same counters and
    decay): a slice of a workload too large to evaluate on the host, or one rank's block of
    auxiliary rows."""
    P = npair(n)
    decay = _tril_decay(n)
    out = np.empty((l1 - l0, P), dtype=np.float64)

    def rows(a: int, b: int) -> None:
        for L in range(a, b):
            out[L - l0] = normals(seed, 0, L * P, P) * decay * np.exp(-L / naux)

    threads = threads or min(32, os.cpu_count() or 1)
    if (l1 - l0) * P < 4_000_000 or threads == 1:
        rows(l0, l1)
    else:
        step = max(1, (l1 - l0 + threads * 4 - 1) // (threads * 4))
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda a: rows(a, min(l1, a + step)), range(l0, l1, step)))
    return out


def one_electron_h(seed: int, n: int) -> np.ndarray:
    z = normals(seed, 1, 0, npair(n)) * _tril_decay(n)
    h = np.zeros((n, n))
    mu, nu = np.tril_indices(n)
    h[mu, nu] = z
    h[nu, mu] = z
    return h


def orthogonal_C(seed: int, n: int) -> np.ndarray:
    g = normals(seed, 2, 0, n * n).reshape(n, n)
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def ci_vector(seed: int, frag: int, m: int, ne: int) -> np.ndarray:
    from .rdm import nstrings
    na = ne // 2
    nb = ne - na
    nsa, nsb = nstrings(m, na), nstrings(m, nb)
    c = normals(seed, 3 + frag, 0, nsa * nsb).reshape(nsa, nsb)
    return c / np.linalg.norm(c)


@dataclass
class LasSystem:
    """One synthetic LAS problem.  MO columns: core, fragment 0, fragment 1, ..., virtuals."""
    nao: int
    naux: int
    nmo: int
    ncore: int
    nact: list[int]
    nelec: list[int]
    seed: int
    Bp: np.ndarray | None = None       # [naux][nao(nao+1)/2] float64
    h: np.ndarray | None = None        # [nao][nao]
    C: np.ndarray | None = None        # [nao][nmo]
    ci: list[np.ndarray] = field(default_factory=list)
    dm1s: list[np.ndarray] = field(default_factory=list)   # per fragment [2][m][m]
    dm2: list[np.ndarray] = field(default_factory=list)    # per fragment [m][m][m][m]

    @property
    def nfrag(self) -> int:
        return len(self.nact)

    @property
    def nactive(self) -> int:
        return int(sum(self.nact))

    @property
    def nocc(self) -> int:
        return self.ncore + self.nactive

    def dm1s_flat(self) -> np.ndarray:
        if not self.dm1s:
            return np.zeros(0)
        return np.concatenate([d.ravel() for d in self.dm1s])

    def dm2_flat(self) -> np.ndarray:
        if not self.dm2:
            return np.zeros(0)
        return np.concatenate([d.ravel() for d in self.dm2])


def make_system(nao: int, naux: int, ncore: int, frags: list[tuple[int, int]], seed: int,
                nmo: int | None = None, with_B: bool = True, threads: int | None = None
                ) -> LasSystem:
    """frags: list of (nelec, norb) per fragment."""
    from .rdm import fragment_rdms
    nmo = nao if nmo is None else nmo
    sysm = LasSystem(nao=nao, naux=naux, nmo=nmo, ncore=ncore,
                     nact=[m for _, m in frags], nelec=[e for e, _ in frags], seed=seed)
    if ncore + sysm.nactive > nmo or nmo > nao:
        raise ValueError("need ncore + sum(nact) <= nmo <= nao")
    if with_B:
        sysm.Bp = packed_B(seed, nao, naux, threads=threads)
    sysm.h = one_electron_h(seed, nao)
    sysm.C = np.ascontiguousarray(orthogonal_C(seed, nao)[:, :nmo])
    for k, (ne, m) in enumerate(frags):
        c = ci_vector(seed, k, m, ne)
        g1, g2 = fragment_rdms(c, m, ne)
        sysm.ci.append(c)
        sysm.dm1s.append(g1)
        sysm.dm2.append(g2)
    return sysm


# Workloads, named by their number of AOs, each with its own seed.
WORKLOADS = {
    "nao48": dict(nao=48, naux=160, ncore=10, frags=[(2, 2), (2, 2)], seed=BASE_SEED),
    "nao400": dict(nao=400, naux=1600, ncore=60, frags=[(4, 4)] * 4, seed=BASE_SEED + 1),
    "nao1200": dict(nao=1200, naux=4800, ncore=150, frags=[(6, 8)] + [(4, 8)] * 4,
                    seed=BASE_SEED + 2),
    "nao800": dict(nao=800, naux=3200, ncore=100, frags=[(6, 6)] * 4, seed=BASE_SEED + 4),
}


def workload_system(name: str, with_B: bool = True, threads: int | None = None) -> LasSystem:
    w = WORKLOADS[name]
    return make_system(w["nao"], w["naux"], w["ncore"], w["frags"], seed=w["seed"],
                       with_B=with_B, threads=threads)


def batched_specs(count: int = 64, seed: int = BASE_SEED + 3) -> list[dict]:
    """Uneven batch: Nao ~ U[100,600], Naux = 4 Nao, Ncore = Nao // 8, 2-6 fragments of 2-8
    orbitals each with 2*floor(m/2) electrons.  Sizes are drawn from stream 1000 of `seed`."""
    u = uniforms(seed, 1000, 0, count * 16)
    specs = []
    for i in range(count):
        r = u[16 * i: 16 * (i + 1)]
        nao = 100 + int(r[0] * 501)
        nfrag = 2 + int(r[1] * 5)
        frags = []
        for k in range(nfrag):
            m = 2 + int(r[2 + k] * 7)
            frags.append((2 * (m // 2), m))
        specs.append(dict(nao=nao, naux=4 * nao, ncore=nao // 8, frags=frags,
                          seed=seed * 1000 + i))
    return specs


def batched_systems(count: int = 64, with_B: bool = True, threads: int | None = None
                    ) -> list[LasSystem]:
    return [make_system(s["nao"], s["naux"], s["ncore"], s["frags"], s["seed"],
                        with_B=with_B, threads=threads) for s in batched_specs(count)]

