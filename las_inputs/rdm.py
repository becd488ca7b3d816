"""Fragment 1- and 2-RDMs from a fragment CI vector (input preparation).

The LAS wave function (Eq. las_wfn) is a product of fragment active-space wave functions and a
core determinant; the energy and gradient kernels consume, per fragment K, the spin-separated
1-RDM gamma^K_sigma[p,q] = <p+_sigma q_sigma> and the spin-summed 2-RDM in chemists' order
Gamma^K[p,q,r,s] = sum_{sigma,tau} <p+_sigma r+_tau s_tau q_sigma> (the quantities D and
gamma_sigma of Eqs. v_emb and vself, and the two-body density that multiplies g in Eq. h_emb).

Determinants are (alpha string, beta string) pairs.  A string is a bit mask over the m fragment
orbitals; strings are enumerated in increasing integer order.  The fermion sign convention is:
all alpha creators, orbital-ascending, to the left of all beta creators, orbital-ascending.
With that convention an alpha excitation p+ q acting on |a, b> only picks up the parity of the
occupied alpha orbitals below q and below p, and a beta excitation only those of the beta
string (the two alpha-string crossings of a beta pair cancel).

The 2-RDM uses the identity  sum_{st} p+_s r+_t s_t q_s = E_pq E_rs - delta_qr E_ps  with the
spin-summed excitation operator E_pq = sum_s p+_s q_s, so
Gamma[p,q,r,s] = <E_qp psi | E_rs psi> - delta_qr D[p,s].
"""
from __future__ import annotations

from functools import lru_cache
from math import comb

import numpy as np


def nstrings(m: int, ne: int) -> int:
    return comb(m, ne)


@lru_cache(maxsize=None)
def strings(m: int, ne: int) -> tuple[int, ...]:
    return tuple(s for s in range(1 << m) if bin(s).count("1") == ne)


def _parity_below(s: int, k: int) -> int:
    return -1 if bin(s & ((1 << k) - 1)).count("1") & 1 else 1


@lru_cache(maxsize=None)
def excitation_matrices(m: int, ne: int) -> np.ndarray:
    """E[p, q] as dense [m][m][nstr][nstr] with <I| p+ q |J> for one spin."""
    strs = strings(m, ne)
    index = {s: i for i, s in enumerate(strs)}
    ns = len(strs)
    E = np.zeros((m, m, ns, ns))
    for j, J in enumerate(strs):
        for q in range(m):
            if not (J >> q) & 1:
                continue
            s1 = _parity_below(J, q)
            Jq = J ^ (1 << q)
            for p in range(m):
                if (Jq >> p) & 1:
                    continue
                s2 = _parity_below(Jq, p)
                I = Jq | (1 << p)
                E[p, q, index[I], j] += s1 * s2
    return E


def fragment_rdms(ci: np.ndarray, m: int, ne: int) -> tuple[np.ndarray, np.ndarray]:
    """Return (dm1s [2][m][m], dm2 [m][m][m][m]) for a real CI vector ci[alpha][beta]."""
    na = ne // 2
    nb = ne - na
    Ea = excitation_matrices(m, na)
    Eb = excitation_matrices(m, nb)
    psi = np.asarray(ci, dtype=np.float64)
    # E^a_pq psi  and  E^b_pq psi as [m][m][nA][nB]
    va = np.einsum("pqij,jk->pqik", Ea, psi)
    vb = np.einsum("pqkj,ij->pqik", Eb, psi)
    ga = np.einsum("ik,pqik->pq", psi, va)
    gb = np.einsum("ik,pqik->pq", psi, vb)
    V = (va + vb).reshape(m, m, -1)
    D = ga + gb
    G = np.einsum("qpx,rsx->pqrs", V, V)
    for q in range(m):
        G[:, q, q, :] -= D
    return np.stack([ga, gb]), G
