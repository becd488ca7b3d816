"""CPU oracle for the density-fitted LAS energy and orbital gradient (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the bench's
CPU-baseline leg may import this module.  The GPU library never calls it and shares no code
with it: the only common module is the seeded input generator ``las_inputs``.

Everything here is written out from the paper's definitions in FP64, with numpy matrix
products (a library primitive) as the only building block beyond plain loops:

* DF factorisation of the two-electron integrals, Eq. cholesky:  g^{mu1 mu3}_{mu2 mu4} =
  b^P_{mu1 mu2} b^P_{mu3 mu4}.  B is stored packed lower-triangular per auxiliary index P
  (index mu(mu+1)/2 + nu, mu >= nu), and unpacked to a square block before use, block by block
  along P as in the paper's JK call (default N_blk = 240, reduced when a block would not fit a
  host-memory budget).
* JK call, Eqs. J_1, J_2, K_1, K_2:  v_P = b^P_ij D_ij ; J_ij = v_P b^P_ij ;
  v^P_ik = b^P_ij gamma_jk ; K_ij = v^P_ik b^P_jk.
* Effective potentials, Eqs. v_emb and vself:  v_sigma = J[D] - K[gamma_sigma], D = sum_sigma
  gamma_sigma (in the AO basis, or in a fragment's embedded basis for the self potential).
* AO2MO, Eqs. ao2mo_1, ao2mo_2, ppaa, papa:  b^P_{e p} = b^P_{ee} M ; b^P_{pp} = b^P_{ep} M ;
  g^{pa}_{pa} = b^P_{pp} b^P_{aa} ; g^{pp}_{aa} = b^P_{pa} b^P_{pa}.
* LAS wave function, Eq. las_wfn: a product of fragment CAS states and a closed-shell core
  determinant.  Its active RDMs are the block products of the fragment RDMs (intra-fragment
  blocks, inter-fragment Coulomb D^K D^L and exchange -sum_sigma gamma^K_sigma gamma^L_sigma).
* LAS energy E_LAS = <LAS|H|LAS> and its derivative with respect to the MO coefficients, the
  quantity behind the orbital-rotation gradient of Eq. MO_conv.  The paper defers these forms
  to its refs. Hermes2019/hermes2020variational; they are written here in the standard
  closed-shell-core form:
      Dc = 2 C_c C_c^T,  Da = C_a D^act C_a^T,
      F^I = h + J[Dc] - K[Dc]/2,   F^A = J[Da] - K[Da]/2,
      E = 1/2 sum Dc (h + F^I) + sum_uv (C_a^T F^I C_a)_uv D_uv + 1/2 sum (uv|wx) Gamma_uvwx,
      dE/dC[:, core] = 4 (F^I + F^A) C_core,
      dE/dC[:, act]  = 2 F^I C_a D^act + 2 sum_vwx (mu v|wx) Gamma_uvwx,
      dE/dC[:, virt] = 0,   g = C^T dE/dC - (C^T dE/dC)^T.
  No nuclear-repulsion constant is included (the paper drops constants, Eq. h_emb).

Tier A (tiny sizes) rebuilds the full MO integrals (pq|rs) and the full-molecule 1-/2-RDMs
and contracts them directly, and a Slater-Condon evaluation of <LAS|H|LAS> over the explicit
product of CI vectors checks the block-product RDMs independently of both.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np

HOST_BLOCK_BYTES = 1 << 30


# ----------------------------------------------------------------------------------------
# Packed Cholesky vectors
# ----------------------------------------------------------------------------------------
def unpack_block(Bp_rows: np.ndarray, n: int) -> np.ndarray:
    """Packed lower triangles [nb][n(n+1)/2] -> symmetric squares [nb][n][n]."""
    nb = Bp_rows.shape[0]
    out = np.zeros((nb, n, n))
    mu, nu = np.tril_indices(n)
    out[:, mu, nu] = Bp_rows
    out[:, nu, mu] = Bp_rows
    return out


def block_size(n: int, naux: int, nblk: int = 240) -> int:
    """Blocks along P of at most N_blk = 240 (the paper's default), smaller if one unpacked
    block would exceed the host-memory budget."""
    fit = max(1, HOST_BLOCK_BYTES // (8 * n * n))
    return max(1, min(nblk, fit, naux))


def p_blocks(Bp: np.ndarray, n: int, l0: int = 0, l1: int | None = None, nblk: int = 240):
    naux = Bp.shape[0]
    l1 = naux if l1 is None else l1
    step = block_size(n, naux, nblk)
    for a in range(l0, l1, step):
        b = min(l1, a + step)
        yield a, b, unpack_block(Bp[a:b], n)


# ----------------------------------------------------------------------------------------
# JK call (Eqs. J_1, J_2, K_1, K_2) and AO2MO (Eqs. ao2mo_1, ao2mo_2, ppaa)
# ----------------------------------------------------------------------------------------
def df_jk(Bp: np.ndarray, n: int, dms: list[np.ndarray], l0: int = 0, l1: int | None = None
          ) -> tuple[list[np.ndarray], list[np.ndarray]]:
    """J[D] and K[D] for each density D (n x n), summed over P in [l0, l1).

    K[D]_ij = sum_P sum_{jk} b^P_ij D_jk b^P_kl is Eq. K_2 applied to the intermediate of
    Eq. K_1 with gamma = D."""
    J = [np.zeros((n, n)) for _ in dms]
    K = [np.zeros((n, n)) for _ in dms]
    for _, _, b in p_blocks(Bp, n, l0, l1):
        for t, D in enumerate(dms):
            nb = b.shape[0]
            vP = b.reshape(nb, n * n) @ D.reshape(n * n)                 # Eq. J_1
            J[t] += (vP @ b.reshape(nb, n * n)).reshape(n, n)           # Eq. J_2
            vPik = b @ D                                                 # Eq. K_1
            K[t] += np.einsum("Pik,Pjk->ij", vPik, b, optimize=True)    # Eq. K_2
    return J, K


def ao2mo_active(Bp: np.ndarray, n: int, C_a: np.ndarray, l0: int = 0, l1: int | None = None
                 ) -> tuple[np.ndarray, np.ndarray]:
    """Returns ((uv|wx) [a]^4, (mu v|wx) [n][a]^3) summed over P in [l0, l1).

    b^P_{mu v} = b^P_{mu nu} C_{nu v} (Eq. ao2mo_1), b^P_{uv} = C_{mu u} b^P_{mu v} (Eq. ao2mo_2),
    and the products b^P_{..} b^P_{wx} (Eq. ppaa) with the first pair left in the AO basis for
    the gradient."""
    a = C_a.shape[1]
    eri = np.zeros((a, a, a, a))
    mveri = np.zeros((n, a, a, a))
    for _, _, b in p_blocks(Bp, n, l0, l1):
        bmv = b @ C_a                                    # Eq. ao2mo_1
        buv = np.einsum("mu,Pmv->Puv", C_a, bmv, optimize=True)  # Eq. ao2mo_2
        nb = b.shape[0]
        eri += (buv.reshape(nb, a * a).T @ buv.reshape(nb, a * a)).reshape(a, a, a, a)  # ppaa
        mveri += np.einsum("Pmv,Pwx->mvwx", bmv, buv, optimize=True)
    return eri, mveri


def df_transform(Bp: np.ndarray, n: int, C: np.ndarray, act: tuple[int, int],
                 p0: int, p1: int) -> tuple[np.ndarray, np.ndarray]:
    """(L|mu u) = sum_nu B_L(mu nu) C(nu,u) for active u, and (L|p u) = sum_mu C(mu,p)(L|mu u)
    for p in [p0, p1) (Eqs. ao2mo_1 and ao2mo_2).  Returns ([X][n][a], [X][p1-p0][a])."""
    C_a = C[:, act[0]:act[1]]
    naux = Bp.shape[0]
    a = C_a.shape[1]
    lmu = np.zeros((naux, n, a))
    lpu = np.zeros((naux, p1 - p0, a))
    for l0, l1, b in p_blocks(Bp, n):
        lmu[l0:l1] = b @ C_a
        lpu[l0:l1] = np.einsum("mp,Pmu->Ppu", C[:, p0:p1], lmu[l0:l1], optimize=True)
    return lmu, lpu


def frag_ao2mo(Bp: np.ndarray, n: int, M: np.ndarray, a0: int, ma: int
               ) -> tuple[np.ndarray, np.ndarray]:
    """Fragment-embedding AO2MO, Eqs. ao2mo_1, ao2mo_2, ppaa and papa, in the basis the
    Cholesky vectors are given in (the fragment's embedded orbitals e).

    b^P_{e2 p1} = b^P_{e1 e2} M_{e1 p1} (Eq. ao2mo_1); b^P_{p1 p2} = b^P_{e2 p1} M_{e2 p2}
    (Eq. ao2mo_2); with the active orbitals a = columns [a0, a0+ma) of M,
    ppaa[p1, p2, a1, a2] = b^P_{p1 p2} b^P_{a1 a2} (Eq. ppaa) and
    papa[p1, a1, p2, a2] = b^P_{p1 a1} b^P_{p2 a2} (Eq. papa), summed over P block by block.
    Returns (ppaa [nmo][nmo][ma][ma], papa [nmo][ma][nmo][ma]) with nmo = M.shape[1]."""
    nmo = M.shape[1]
    act = slice(a0, a0 + ma)
    ppaa = np.zeros((nmo, nmo, ma, ma))
    papa = np.zeros((nmo, ma, nmo, ma))
    for _, _, b in p_blocks(Bp, n):
        nb = b.shape[0]
        bep = b @ M                                                   # Eq. ao2mo_1
        bpp = np.einsum("ep,Peq->Ppq", M, bep, optimize=True)         # Eq. ao2mo_2
        baa = bpp[:, act, act]
        ppaa += (bpp.reshape(nb, nmo * nmo).T @ baa.reshape(nb, ma * ma)
                 ).reshape(nmo, nmo, ma, ma)                          # Eq. ppaa
        bpa = bpp[:, :, act].reshape(nb, nmo * ma)
        papa += (bpa.T @ bpa).reshape(nmo, ma, nmo, ma)               # Eq. papa
    return ppaa, papa


def embedding_potentials(Bp: np.ndarray, n: int, gam_a: np.ndarray, gam_b: np.ndarray
                         ) -> tuple[np.ndarray, np.ndarray]:
    """Effective potentials of Eq. v_emb (or of Eq. vself when B and the densities are given in
    a fragment's embedded basis): v_sigma = g^{..}_{..} D - g^{..}_{..} gamma_sigma, i.e.
    v_sigma = J[gamma_alpha + gamma_beta] - K[gamma_sigma] with J and K of the JK call
    (Eqs. J_1-K_2).  Returns (v_alpha, v_beta)."""
    (J_a, J_b), (K_a, K_b) = df_jk(Bp, n, [gam_a, gam_b])
    J = J_a + J_b
    return J - K_a, J - K_b


# ----------------------------------------------------------------------------------------
# Block-product active RDMs of the LAS state (Eq. las_wfn)
# ----------------------------------------------------------------------------------------
def active_rdms(dm1s: list[np.ndarray], dm2: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """D^act [a][a] and Gamma^act [a]^4 from per-fragment (gamma_a, gamma_b) and Gamma^K."""
    sizes = [d.shape[-1] for d in dm1s]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    a = int(offs[-1])
    D = np.zeros((a, a))
    G = np.zeros((a, a, a, a))
    for K, (g1, g2) in enumerate(zip(dm1s, dm2)):
        sK = slice(offs[K], offs[K + 1])
        D[sK, sK] = g1[0] + g1[1]
        G[sK, sK, sK, sK] = g2
    for K, L in product(range(len(sizes)), repeat=2):
        if K == L:
            continue
        sK = slice(offs[K], offs[K + 1])
        sL = slice(offs[L], offs[L + 1])
        DK = dm1s[K][0] + dm1s[K][1]
        DL = dm1s[L][0] + dm1s[L][1]
        # Gamma[p,q,r,s] = D^K_pq D^L_rs                       (p,q in K; r,s in L)
        G[sK, sK, sL, sL] = np.einsum("pq,rs->pqrs", DK, DL)
        # Gamma[p,s,r,q] = -sum_sigma g^K_sigma[p,q] g^L_sigma[r,s]
        ex = -sum(np.einsum("pq,rs->pqrs", dm1s[K][s], dm1s[L][s]) for s in range(2))
        G[sK, sL, sL, sK] = ex.transpose(0, 3, 2, 1)
    return D, G


# ----------------------------------------------------------------------------------------
# Tier B: energy and gradient through J/K (all sizes)
# ----------------------------------------------------------------------------------------
def _fsum_dot(a: np.ndarray, b: np.ndarray) -> float:
    return math.fsum((np.asarray(a) * np.asarray(b)).ravel())


def energy_grad(Bp: np.ndarray, n: int, h: np.ndarray, C: np.ndarray, ncore: int,
                dm1s: list[np.ndarray], dm2: list[np.ndarray], with_grad: bool = True,
                l0: int = 0, l1: int | None = None) -> dict:
    """LAS energy and dE/dC (n x nmo).  With (l0, l1) only auxiliary rows P in [l0, l1)
    contribute to the two-electron part (a bounded sample for timing)."""
    nact = [d.shape[-1] for d in dm1s]
    a = int(sum(nact))
    C_c = C[:, :ncore]
    C_a = C[:, ncore:ncore + a]
    Dact, Gact = active_rdms(dm1s, dm2) if a else (np.zeros((0, 0)), np.zeros((0,) * 4))
    Dc = 2.0 * C_c @ C_c.T
    Da = C_a @ Dact @ C_a.T
    (Jc, Ja), (Kc, Ka) = df_jk(Bp, n, [Dc, Da], l0, l1)
    FI = h + Jc - 0.5 * Kc
    FA = Ja - 0.5 * Ka
    heff = C_a.T @ FI @ C_a
    if a:
        eri, mveri = ao2mo_active(Bp, n, C_a, l0, l1)
    else:
        eri, mveri = np.zeros((0,) * 4), np.zeros((n, 0, 0, 0))
    e_core = 0.5 * _fsum_dot(Dc, h + FI)
    e_act1 = _fsum_dot(heff, Dact)
    e_act2 = 0.5 * _fsum_dot(eri, Gact)
    out = dict(E=e_core + e_act1 + e_act2, e_core=e_core, e_act1=e_act1, e_act2=e_act2,
               J=Jc, K=Kc, Ja=Ja, Ka=Ka, FI=FI, FA=FA, eri=eri, Dact=Dact, Gact=Gact)
    if with_grad:
        G = np.zeros_like(C)
        G[:, :ncore] = 4.0 * (FI + FA) @ C_c
        if a:
            G[:, ncore:ncore + a] = 2.0 * FI @ C_a @ Dact + 2.0 * np.einsum(
                "mvwx,uvwx->mu", mveri, Gact, optimize=True)
        CtG = C.T @ G
        out.update(G=G, Fgen=0.5 * CtG, gorb=CtG - CtG.T)
    return out


def grad_derivative(Bp: np.ndarray, n: int, h: np.ndarray, C: np.ndarray, ncore: int,
                    dm1s: list[np.ndarray], dm2: list[np.ndarray], dC: np.ndarray) -> dict:
    """Directional derivative of dE/dC along dC at fixed fragment RDMs: the linearisation of
    the gradient formulas of `energy_grad` term by term,
        dDc = 2 (dC_c C_c^T + C_c dC_c^T),   dDa = dC_a D C_a^T + C_a D dC_a^T,
        dF^I = J[dDc] - K[dDc]/2,            dF^A = J[dDa] - K[dDa]/2,
        dG[:, core] = 4 (dF^I + dF^A) C_c + 4 (F^I + F^A) dC_c,
        dG[:, act]  = 2 dF^I C_a D + 2 F^I dC_a D + 2 sum_vwx d(mu v|wx) Gamma_uvwx,
        d(mu v|wx)  = sum_P (b^P dC_a)_{mu v} (C_a^T b^P C_a)_wx
                      + (b^P C_a)_{mu v} (dC_a^T b^P C_a + C_a^T b^P dC_a)_wx.
    Returns G, dG (n x nmo) and the matching quantities of the orbital-rotation gradient."""
    nact = [d.shape[-1] for d in dm1s]
    a = int(sum(nact))
    C_c, C_a = C[:, :ncore], C[:, ncore:ncore + a]
    dC_c, dC_a = dC[:, :ncore], dC[:, ncore:ncore + a]
    Dact, Gact = active_rdms(dm1s, dm2) if a else (np.zeros((0, 0)), np.zeros((0,) * 4))
    Dc = 2.0 * C_c @ C_c.T
    Da = C_a @ Dact @ C_a.T
    dDc = 2.0 * (dC_c @ C_c.T + C_c @ dC_c.T)
    dDa = dC_a @ Dact @ C_a.T + C_a @ Dact @ dC_a.T
    (Jc, Ja, dJc, dJa), (Kc, Ka, dKc, dKa) = df_jk(Bp, n, [Dc, Da, dDc, dDa])
    FI, FA = h + Jc - 0.5 * Kc, Ja - 0.5 * Ka
    dFI, dFA = dJc - 0.5 * dKc, dJa - 0.5 * dKa
    G = np.zeros_like(C)
    dG = np.zeros_like(C)
    G[:, :ncore] = 4.0 * (FI + FA) @ C_c
    dG[:, :ncore] = 4.0 * (dFI + dFA) @ C_c + 4.0 * (FI + FA) @ dC_c
    if a:
        mveri = np.zeros((n, a, a, a))
        dmveri = np.zeros((n, a, a, a))
        for _, _, b in p_blocks(Bp, n):
            bmv = b @ C_a                                            # (b^P C_a)_{mu v}
            dbmv = b @ dC_a
            buv = np.einsum("mu,Pmv->Puv", C_a, bmv, optimize=True)  # C_a^T b^P C_a
            dbuv = np.einsum("mu,Pmv->Puv", dC_a, bmv, optimize=True)
            dbuv = dbuv + dbuv.transpose(0, 2, 1)                    # b^P symmetric
            mveri += np.einsum("Pmv,Pwx->mvwx", bmv, buv, optimize=True)
            dmveri += (np.einsum("Pmv,Pwx->mvwx", dbmv, buv, optimize=True)
                       + np.einsum("Pmv,Pwx->mvwx", bmv, dbuv, optimize=True))
        G[:, ncore:ncore + a] = 2.0 * FI @ C_a @ Dact + 2.0 * np.einsum(
            "mvwx,uvwx->mu", mveri, Gact, optimize=True)
        dG[:, ncore:ncore + a] = (2.0 * dFI @ C_a @ Dact + 2.0 * FI @ dC_a @ Dact
                                  + 2.0 * np.einsum("mvwx,uvwx->mu", dmveri, Gact,
                                                    optimize=True))
    return dict(G=G, dG=dG)


def orbital_hvp(Bp: np.ndarray, n: int, h: np.ndarray, C: np.ndarray, ncore: int,
                dm1s: list[np.ndarray], dm2: list[np.ndarray], X: np.ndarray) -> dict:
    """Derivative of the orbital-rotation gradient g(C) = C^T G - (C^T G)^T along the rotation
    C(t) = C exp(t X) at t = 0 (X antisymmetric, nmo x nmo), at fixed fragment RDMs:
        Dg = (C X)^T G + C^T dG - transpose,   dG = dE/dC differentiated along dC = C X."""
    dC = C @ X
    r = grad_derivative(Bp, n, h, C, ncore, dm1s, dm2, dC)
    M = dC.T @ r["G"] + C.T @ r["dG"]
    return dict(G=r["G"], dG=r["dG"], dC=dC, Dg=M - M.T)


def system_energy_grad(sysm, with_grad: bool = True, l0: int = 0, l1: int | None = None) -> dict:
    return energy_grad(sysm.Bp, sysm.nao, sysm.h, sysm.C, sysm.ncore, sysm.dm1s, sysm.dm2,
                       with_grad=with_grad, l0=l0, l1=l1)


# ----------------------------------------------------------------------------------------
# Tier A: explicit MO integrals and full-molecule RDMs (tiny sizes only)
# ----------------------------------------------------------------------------------------
def mo_eri(Bp: np.ndarray, n: int, Cocc: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_P (C^T b^P C)_pq (C^T b^P C)_rs over the given MO columns."""
    b = unpack_block(Bp, n)
    t = np.einsum("mp,Pmn,nq->Ppq", Cocc, b, Cocc)
    return np.einsum("Ppq,Prs->pqrs", t, t)


def full_rdms(ncore: int, Dact: np.ndarray, Gact: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """1- and 2-RDM over core+active MOs of (closed-shell core) x (active state)."""
    c = ncore
    a = Dact.shape[0]
    o = c + a
    D = np.zeros((o, o))
    G = np.zeros((o, o, o, o))
    for i in range(c):
        D[i, i] = 2.0
        for j in range(c):
            G[i, i, j, j] += 4.0
            G[i, j, j, i] -= 2.0
    act = slice(c, o)
    D[act, act] = Dact
    G[act, act, act, act] = Gact
    for i in range(c):
        G[i, i, act, act] += 2.0 * Dact
        G[act, act, i, i] += 2.0 * Dact
        G[i, act, act, i] -= Dact
        G[act, i, i, act] -= Dact
    return D, G


def energy_tier_a(Bp: np.ndarray, n: int, h: np.ndarray, C: np.ndarray, ncore: int,
                  dm1s: list[np.ndarray], dm2: list[np.ndarray]) -> float:
    a = int(sum(d.shape[-1] for d in dm1s))
    Cocc = C[:, :ncore + a]
    Dact, Gact = active_rdms(dm1s, dm2) if a else (np.zeros((0, 0)), np.zeros((0,) * 4))
    D, G = full_rdms(ncore, Dact, Gact)
    hmo = Cocc.T @ h @ Cocc
    eri = mo_eri(Bp, n, Cocc)
    return _fsum_dot(hmo, D) + 0.5 * _fsum_dot(eri, G)


def ao_eri(Bp: np.ndarray, n: int) -> np.ndarray:
    """Brute-force 4-index (mu nu|la si) = sum_P b^P_{mu nu} b^P_{la si} (Eq. cholesky)."""
    b = unpack_block(Bp, n)
    return np.einsum("Pmn,Pls->mnls", b, b)


# ----------------------------------------------------------------------------------------
# Slater-Condon evaluation of <LAS|H|LAS> over the explicit product CI vector
# ----------------------------------------------------------------------------------------
def _perm_parity(seq: list[int]) -> int:
    inv = 0
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                inv += 1
    return -1 if inv & 1 else 1


def _sign_apply(occ_bits: int, k: int) -> int:
    return -1 if bin(occ_bits & ((1 << k) - 1)).count("1") & 1 else 1


def product_determinants(ncore: int, nact: list[int], nelec: list[int], cis: list[np.ndarray]):
    """Expand (wedge_K Psi_K) ^ core into determinants over o = ncore + a spatial orbitals.

    Spin orbital index: alpha k -> k, beta k -> o + k.  A determinant is the product of its
    creators in increasing spin-orbital order.  The wedge product is taken in the order
    fragment 0 (alpha string then beta string), fragment 1, ..., core alpha, core beta; the sign
    of each expanded determinant is the parity of sorting that creator sequence."""
    from las_inputs.rdm import strings
    o = ncore + sum(nact)
    offs = np.concatenate([[ncore], ncore + np.cumsum(nact)]).astype(int)
    per_frag = []
    for K, (m, ne) in enumerate(zip(nact, nelec)):
        na = ne // 2
        nb = ne - na
        sa, sb = strings(m, na), strings(m, nb)
        items = []
        for ia, A in enumerate(sa):
            for ib, Bs in enumerate(sb):
                ca = [offs[K] + k for k in range(m) if (A >> k) & 1]
                cb = [o + offs[K] + k for k in range(m) if (Bs >> k) & 1]
                items.append((cis[K][ia, ib], ca + cb))
        per_frag.append(items)
    core = list(range(ncore)) + [o + i for i in range(ncore)]
    dets = {}
    for combo in product(*per_frag):
        coef = 1.0
        seq = []
        for cK, ops in combo:
            coef *= cK
            seq += ops
        seq += core
        sign = _perm_parity(seq)
        bits = 0
        for k in seq:
            bits |= 1 << k
        dets[bits] = dets.get(bits, 0.0) + sign * coef
    return o, dets


def slater_condon_energy(hmo: np.ndarray, eri: np.ndarray, o: int, dets: dict) -> float:
    """sum_IJ c_I c_J <I|H|J> with the Slater-Condon rules in spin orbitals, where
    h_{pq} and [pq|rs] = (pq|rs) vanish unless the paired spins agree."""
    def sp(k):
        return k % o, k // o

    def hso(p, q):
        (pp, ps), (qq, qs) = sp(p), sp(q)
        return hmo[pp, qq] if ps == qs else 0.0

    def gso(p, q, r, s):
        (pp, ps), (qq, qs), (rr, rs), (ss, sss) = sp(p), sp(q), sp(r), sp(s)
        if ps != qs or rs != sss:
            return 0.0
        return eri[pp, qq, rr, ss]

    keys = list(dets)
    total = []
    for I in keys:
        occI = [k for k in range(2 * o) if (I >> k) & 1]
        for J in keys:
            x = I ^ J
            nd = bin(x).count("1")
            if nd > 4:
                continue
            cij = dets[I] * dets[J]
            if nd == 0:
                e = sum(hso(k, k) for k in occI)
                e += 0.5 * sum(gso(k, k, l, l) - gso(k, l, l, k) for k in occI for l in occI)
            elif nd == 2:
                m = [k for k in range(2 * o) if (J >> k) & 1 and not (I >> k) & 1][0]
                p = [k for k in range(2 * o) if (I >> k) & 1 and not (J >> k) & 1][0]
                s1 = _sign_apply(J, m)
                Jm = J ^ (1 << m)
                s2 = _sign_apply(Jm, p)
                occJ = [k for k in range(2 * o) if (J >> k) & 1 and k != m]
                e = s1 * s2 * (hso(p, m) + sum(gso(p, m, k, k) - gso(p, k, k, m) for k in occJ))
            else:
                ms = [k for k in range(2 * o) if (J >> k) & 1 and not (I >> k) & 1]
                ps = [k for k in range(2 * o) if (I >> k) & 1 and not (J >> k) & 1]
                m, nn = ms
                p, q = ps
                # |I> = sign a+_p a+_q a_n a_m |J>
                bits = J
                sign = _sign_apply(bits, m)
                bits ^= 1 << m
                sign *= _sign_apply(bits, nn)
                bits ^= 1 << nn
                sign *= _sign_apply(bits, q)
                bits |= 1 << q
                sign *= _sign_apply(bits, p)
                e = sign * (gso(p, m, q, nn) - gso(p, nn, q, m))
            total.append(cij * e)
    return math.fsum(total)


def energy_slater_condon(sysm) -> float:
    a = sysm.nactive
    Cocc = sysm.C[:, :sysm.ncore + a]
    hmo = Cocc.T @ sysm.h @ Cocc
    eri = mo_eri(sysm.Bp, sysm.nao, Cocc)
    o, dets = product_determinants(sysm.ncore, sysm.nact, sysm.nelec, sysm.ci)
    return slater_condon_energy(hmo, eri, o, dets)
