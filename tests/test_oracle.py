"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check below is chosen so that a plausible slip in the oracle (a dropped factor, a wrong
exchange sign, a transposed operand) fails at least one of them; test_planted_mistakes plants
such slips and confirms that they are caught.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from las_inputs import workload_system, make_system, splitmix64
from las_inputs.rdm import fragment_rdms, nstrings, strings
from oracle import las_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def nao48():
    return workload_system("nao48")


@pytest.fixture(scope="module")
def small3():
    # three fragments of different size, one with an odd electron count (Ms = 1/2)
    return make_system(14, 40, 3, [(2, 2), (3, 3), (2, 3)], seed=777)


def test_splitmix64_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if ln.strip() and not ln.startswith("#")]
    gamma = np.uint64(0x9E3779B97F4A7C15)
    for i, ref in rows:
        got = int(splitmix64(np.array([int(i)], dtype=np.uint64) * gamma)[0])
        assert got == int(ref, 16)


def test_generator_properties(nao48):
    s = nao48
    assert np.abs(s.C.T @ s.C - np.eye(s.nmo)).max() < 1e-13
    assert np.allclose(s.h, s.h.T)
    # B decays along L as exp(-L/Naux): compare mean squares of first and last quarters
    q = s.naux // 4
    r = np.mean(s.Bp[-q:] ** 2) / np.mean(s.Bp[:q] ** 2)
    expect = np.mean(np.exp(-2 * np.arange(s.naux - q, s.naux) / s.naux)) / np.mean(
        np.exp(-2 * np.arange(q) / s.naux))
    assert abs(r / expect - 1) < 0.1


def test_unpack_block_packed_index_convention():
    """The packed layout of the Cholesky vectors (lower triangle per auxiliary index, section
    "Calculation of effective potentials"): element mu(mu+1)/2 + nu, mu >= nu, is b_{mu nu} and,
    by symmetry, b_{nu mu}.  Written out by hand for n = 3 so that a row-order slip (the upper
    triangle's order, or nu(nu+1)/2 + mu) cannot hide behind numpy's index helpers."""
    row = np.array([[10.0, 21.0, 22.0, 31.0, 32.0, 33.0]])   # b00 b10 b11 b20 b21 b22
    expect = np.array([[10.0, 21.0, 31.0],
                       [21.0, 22.0, 32.0],
                       [31.0, 32.0, 33.0]])
    assert np.array_equal(O.unpack_block(row, 3)[0], expect)
    # n = 4, one auxiliary row per element: only (mu, nu) and (nu, mu) are hit
    n = 4
    P = n * (n + 1) // 2
    for mu in range(n):
        for nu in range(mu + 1):
            one = np.zeros((1, P))
            one[0, mu * (mu + 1) // 2 + nu] = 1.0
            sq = O.unpack_block(one, n)[0]
            hit = np.zeros((n, n))
            hit[mu, nu] = hit[nu, mu] = 1.0
            assert np.array_equal(sq, hit), (mu, nu)


def test_unpacked_generator_band(nao48):
    """Unpacked, the seeded Cholesky vectors show the band of the generator recipe,
    rms of b_{mu nu} over (L, mu) falling as exp(-|mu - nu|/8): a packed-index slip in the
    oracle's unpacking would scramble the band."""
    s = nao48
    b = O.unpack_block(s.Bp, s.nao)
    w = np.exp(-np.arange(s.naux) / s.naux)
    b = b / w[:, None, None]                        # remove the decay along L
    rms = [np.sqrt(np.mean(np.diagonal(b, offset=d, axis1=1, axis2=2) ** 2))
           for d in range(0, 25)]
    for d in range(25):
        assert abs(rms[d] / rms[0] - math.exp(-d / 8.0)) < 0.08 * math.exp(-d / 8.0), d


def test_rdm_sum_rules():
    for ne, m in [(2, 2), (4, 4), (6, 8), (3, 3), (6, 6)]:
        from las_inputs.gen import ci_vector
        ci = ci_vector(99, 0, m, ne)
        g1, g2 = fragment_rdms(ci, m, ne)
        na, nb = ne // 2, ne - ne // 2
        assert abs(np.trace(g1[0]) - na) < 1e-12
        assert abs(np.trace(g1[1]) - nb) < 1e-12
        D = g1[0] + g1[1]
        assert np.abs(np.einsum("pqrr->pq", g2) - (ne - 1) * D).max() < 1e-12
        assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-12      # pair swap
        assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-12      # hermiticity (real)
        w = np.linalg.eigvalsh(D)
        assert w.min() > -1e-12 and w.max() < 2 + 1e-12
        assert abs(np.einsum("pprr->", g2) - ne * (ne - 1)) < 1e-10


def test_rdm_one_hot_determinant():
    m, ne = 4, 4
    na = nb = 2
    sa, sb = strings(m, na), strings(m, nb)
    ci = np.zeros((nstrings(m, na), nstrings(m, nb)))
    ia, ib = 2, 4
    ci[ia, ib] = 1.0
    g1, g2 = fragment_rdms(ci, m, ne)
    occa = np.array([(sa[ia] >> k) & 1 for k in range(m)], float)
    occb = np.array([(sb[ib] >> k) & 1 for k in range(m)], float)
    assert np.allclose(g1[0], np.diag(occa)) and np.allclose(g1[1], np.diag(occb))
    # single determinant: Gamma_pqrs = d_pq d_rs n_p n_r - d_ps d_qr sum_s n_ps n_qs
    n = occa + occb
    I = np.eye(m)
    ref = np.einsum("pq,rs,p,r->pqrs", I, I, n, n) - np.einsum(
        "ps,qr,pq->pqrs", I, I, np.outer(occa, occa) + np.outer(occb, occb))
    assert np.abs(g2 - ref).max() < 1e-14


def test_df_jk_brute_force():
    s = make_system(10, 30, 2, [(2, 2)], seed=5)
    n = s.nao
    eri = O.ao_eri(s.Bp, n)
    rng = np.random.default_rng(0)
    D = rng.standard_normal((n, n))
    D = D + D.T
    (J,), (K,) = O.df_jk(s.Bp, n, [D])
    assert np.abs(J - np.einsum("mnls,ls->mn", eri, D)).max() < 1e-12
    assert np.abs(K - np.einsum("mlsn,ls->mn", eri, D)).max() < 1e-12
    # 8-fold symmetry of the AO integrals built from the factorisation
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(eri - eri.transpose(perm)).max() < 1e-13


def test_active_integral_symmetry(nao48):
    s = nao48
    a = s.nactive
    C_a = s.C[:, s.ncore:s.ncore + a]
    eri, mveri = O.ao2mo_active(s.Bp, s.nao, C_a)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.abs(eri - eri.transpose(perm)).max() < 1e-12
    # (mu v|wx) projected with C_a gives (uv|wx); (pu|vw) has its 4-fold symmetry in (v,w)
    assert np.abs(np.einsum("mu,mvwx->uvwx", C_a, mveri) - eri).max() < 1e-12
    assert np.abs(mveri - mveri.transpose(0, 1, 3, 2)).max() < 1e-12
    # the same integrals straight from the full MO brute force
    full = O.mo_eri(s.Bp, s.nao, C_a)
    assert np.abs(full - eri).max() < 1e-12


def test_df_transform_matches_mo_integrals(nao48):
    s = nao48
    a0, a1 = s.ncore, s.ncore + s.nactive
    lmu, lpu = O.df_transform(s.Bp, s.nao, s.C, (a0, a1), 0, s.nmo)
    b = O.unpack_block(s.Bp, s.nao)
    assert np.abs(lmu - np.einsum("Pmn,nu->Pmu", b, s.C[:, a0:a1])).max() < 1e-12
    # (pu|vw) = sum_L (L|pu)(L|vw) equals the brute-force MO integrals
    pu_vw = np.einsum("Lpu,Lvw->puvw", lpu, lpu[:, a0:a1, :])
    full = O.mo_eri(s.Bp, s.nao, s.C)
    assert np.abs(pu_vw - full[:, a0:a1, a0:a1, a0:a1]).max() < 1e-11


def _frag_case():
    # a non-orthogonal embedded-orbital matrix M (the transform need not be unitary)
    s = make_system(9, 26, 2, [(2, 2)], seed=31)
    rng = np.random.default_rng(7)
    M = rng.standard_normal((s.nao, s.nao))
    return s, M, 3, 3


def test_frag_ao2mo_brute_force():
    """Eqs. ao2mo_1..papa against the 4-index AO integrals transformed index by index."""
    s, M, a0, ma = _frag_case()
    ppaa, papa = O.frag_ao2mo(s.Bp, s.nao, M, a0, ma)
    eri = np.einsum("mnls,mp,nq,lr,st->pqrt", O.ao_eri(s.Bp, s.nao), M, M, M, M)
    act = slice(a0, a0 + ma)
    assert np.abs(ppaa - eri[:, :, act, act]).max() < 1e-10 * np.abs(eri).max()
    assert np.abs(papa - eri[:, act, :, act]).max() < 1e-10 * np.abs(eri).max()


def test_frag_ao2mo_symmetry_and_consistency():
    s, M, a0, ma = _frag_case()
    ppaa, papa = O.frag_ao2mo(s.Bp, s.nao, M, a0, ma)
    act = slice(a0, a0 + ma)
    tol = 1e-12 * np.abs(ppaa).max()
    assert np.abs(ppaa - ppaa.transpose(1, 0, 2, 3)).max() < tol
    assert np.abs(ppaa - ppaa.transpose(0, 1, 3, 2)).max() < tol
    assert np.abs(papa - papa.transpose(2, 3, 0, 1)).max() < tol
    # (P a_k|a_i a_j) appears in both outputs
    assert np.abs(ppaa[:, act, :, :] - papa[:, :, act, :]).max() < tol
    # (pa|pa) from the half/full transform of Eqs. ao2mo_1-ao2mo_2 written the other way round
    _, lpu = O.df_transform(s.Bp, s.nao, M, (a0, a0 + ma), 0, s.nao)
    assert np.abs(np.einsum("Lpu,Lqv->puqv", lpu, lpu) - papa).max() < tol
    # a transposed M (a plausible slip) fails the brute-force pin
    bad, _ = O.frag_ao2mo(s.Bp, s.nao, np.ascontiguousarray(M.T), a0, ma)
    eri = np.einsum("mnls,mp,nq,lr,st->pqrt", O.ao_eri(s.Bp, s.nao), M, M, M, M)
    assert np.abs(bad - eri[:, :, act, act]).max() > 1e-3 * np.abs(eri).max()


def _spin_densities(s):
    """gamma_sigma = C_c C_c^T + C_a gamma^act_sigma C_a^T of a LAS state (AO basis)."""
    c, a = s.ncore, s.nactive
    C_c, C_a = s.C[:, :c], s.C[:, c:c + a]
    out = []
    for sigma in range(2):
        g = np.zeros((a, a))
        off = 0
        for d in s.dm1s:
            m = d.shape[-1]
            g[off:off + m, off:off + m] = d[sigma]
            off += m
        out.append(C_c @ C_c.T + C_a @ g @ C_a.T)
    return out


def test_embedding_potentials_brute_force(small3):
    """Eq. v_emb with the 4-index integrals written out (open-shell fragment: gamma_a != gamma_b)."""
    s = small3
    ga, gb = _spin_densities(s)
    assert np.abs(ga - gb).max() > 1e-3
    va, vb = O.embedding_potentials(s.Bp, s.nao, ga, gb)
    eri = O.ao_eri(s.Bp, s.nao)
    D = ga + gb
    for v, g in ((va, ga), (vb, gb)):
        ref = np.einsum("mnls,ls->mn", eri, D) - np.einsum("mlsn,ls->mn", eri, g)
        assert np.abs(v - ref).max() < 1e-11 * np.abs(ref).max()
    # a plausible slip, the other spin's exchange, is caught
    ref_a = np.einsum("mnls,ls->mn", eri, D) - np.einsum("mlsn,ls->mn", eri, ga)
    assert np.abs(vb - ref_a).max() > 1e-6 * np.abs(ref_a).max()


def test_embedding_potentials_match_fock_terms(small3):
    """Closed-shell core alone: v_sigma = F^I - h; the LAS state: (v_a + v_b)/2 = F^I - h + F^A
    (the Fock-like matrices of the pinned energy and gradient)."""
    s = small3
    r = O.system_energy_grad(s, with_grad=False)
    C_c = s.C[:, :s.ncore]
    gc = C_c @ C_c.T
    va, vb = O.embedding_potentials(s.Bp, s.nao, gc, gc)
    ref = r["FI"] - s.h
    assert np.abs(va - ref).max() < 1e-11 * np.abs(ref).max()
    assert np.abs(vb - ref).max() < 1e-11 * np.abs(ref).max()
    ga, gb = _spin_densities(s)
    va, vb = O.embedding_potentials(s.Bp, s.nao, ga, gb)
    ref = r["FI"] - s.h + r["FA"]
    assert np.abs(0.5 * (va + vb) - ref).max() < 1e-11 * np.abs(ref).max()


def _directions(s, seed, k=2):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        X = rng.standard_normal((s.nmo, s.nmo))
        out.append((X - X.T) / np.sqrt(2.0))
    return out


def _egrad(s, C):
    return O.energy_grad(s.Bp, s.nao, s.h, C, s.ncore, s.dm1s, s.dm2)


def test_grad_derivative_symmetric_and_exact_on_the_energy(small3):
    """<dC2, dG(dC1)> = <dC1, dG(dC2)> (the Hessian of E(C) is symmetric), and along a line
    E(C + t dC) is a quartic, so the five-point stencils give E'(0) and E''(0) exactly:
    E'(0) = <G, dC>, E''(0) = <dC, dG(dC)>."""
    s = small3
    rng = np.random.default_rng(11)
    dC1, dC2 = rng.standard_normal(s.C.shape), rng.standard_normal(s.C.shape)
    r1 = O.grad_derivative(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, dC1)
    r2 = O.grad_derivative(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, dC2)
    a12, a21 = np.sum(dC2 * r1["dG"]), np.sum(dC1 * r2["dG"])
    assert abs(a12 - a21) <= 1e-10 * max(abs(a12), 1.0)
    tau = 0.05
    E = {t: _egrad(s, s.C + t * tau * dC1)["E"] for t in (-2, -1, 0, 1, 2)}
    d1 = (E[-2] - 8 * E[-1] + 8 * E[1] - E[2]) / (12 * tau)
    d2 = (-E[-2] + 16 * E[-1] - 30 * E[0] + 16 * E[1] - E[2]) / (12 * tau * tau)
    assert abs(d1 - np.sum(r1["G"] * dC1)) <= 1e-8 * abs(d1)
    assert abs(d2 - np.sum(dC1 * r1["dG"])) <= 1e-7 * abs(d2)


def test_grad_derivative_finite_differences(nao48):
    s = nao48
    dC = np.random.default_rng(12).standard_normal(s.C.shape)
    r = O.grad_derivative(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, dC)
    eps = 1e-4
    fd = (_egrad(s, s.C + eps * dC)["G"] - _egrad(s, s.C - eps * dC)["G"]) / (2 * eps)
    assert np.abs(fd - r["dG"]).max() <= 1e-6 * np.abs(r["dG"]).max()


def test_orbital_hvp_finite_differences(small3):
    """Dg against central differences of g(C exp(t X))."""
    s = small3
    for X in _directions(s, 13):
        r = O.orbital_hvp(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2, X)
        eps = 1e-5
        gp = _egrad(s, s.C @ sl.expm(eps * X))["gorb"]
        gm = _egrad(s, s.C @ sl.expm(-eps * X))["gorb"]
        fd = (gp - gm) / (2 * eps)
        assert np.abs(fd - r["Dg"]).max() <= 1e-6 * np.abs(r["Dg"]).max()
        assert np.abs(r["Dg"] + r["Dg"].T).max() <= 1e-12 * np.abs(r["Dg"]).max()


@pytest.mark.parametrize("which", ["nao48", "small3"])
def test_energy_three_ways(which, request):
    s = request.getfixturevalue(which)
    eb = O.system_energy_grad(s, with_grad=False)["E"]
    ea = O.energy_tier_a(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2)
    esc = O.energy_slater_condon(s)
    assert abs(ea - eb) < 1e-12 * max(1, abs(eb))
    assert abs(esc - eb) < 1e-12 * max(1, abs(eb))


def test_one_hot_ci_closed_form():
    s = make_system(12, 36, 2, [(2, 2), (4, 3)], seed=31)
    # replace CI vectors by single determinants and rebuild the RDMs
    occ_sets = []
    for K, (ne, m) in enumerate(zip(s.nelec, s.nact)):
        na, nb = ne // 2, ne - ne // 2
        ci = np.zeros((nstrings(m, na), nstrings(m, nb)))
        ci[-1, 0] = 1.0
        s.ci[K] = ci
        s.dm1s[K], s.dm2[K] = fragment_rdms(ci, m, ne)
        off = s.ncore + sum(s.nact[:K])
        sa, sb = strings(m, na)[-1], strings(m, nb)[0]
        occ_sets += [(off + k, 0) for k in range(m) if (sa >> k) & 1]
        occ_sets += [(off + k, 1) for k in range(m) if (sb >> k) & 1]
    occ_sets += [(i, sp) for i in range(s.ncore) for sp in (0, 1)]
    a = s.nactive
    Cocc = s.C[:, :s.ncore + a]
    hmo = Cocc.T @ s.h @ Cocc
    eri = O.mo_eri(s.Bp, s.nao, Cocc)
    e = sum(hmo[i, i] for i, _ in occ_sets)
    e += 0.5 * sum(eri[i, i, j, j] - (eri[i, j, j, i] if si == sj else 0.0)
                   for i, si in occ_sets for j, sj in occ_sets)
    eb = O.system_energy_grad(s, with_grad=False)["E"]
    assert abs(e - eb) < 1e-12 * max(1, abs(e))


def test_no_fragments_rhf():
    s = make_system(16, 48, 4, [], seed=11)
    r = O.system_energy_grad(s)
    Cc = s.C[:, :4]
    hmo = Cc.T @ s.h @ Cc
    eri = O.mo_eri(s.Bp, s.nao, Cc)
    e = 2 * np.trace(hmo) + 2 * np.einsum("iijj->", eri) - np.einsum("ijji->", eri)
    assert abs(r["E"] - e) < 1e-12 * max(1, abs(e))
    # core columns of dE/dC are 4 F^I C_core; F^I from the brute-force AO integrals
    aoeri = O.ao_eri(s.Bp, s.nao)
    Dc = 2 * Cc @ Cc.T
    FI = s.h + np.einsum("mnls,ls->mn", aoeri, Dc) - 0.5 * np.einsum("mlsn,ls->mn", aoeri, Dc)
    assert np.abs(r["G"][:, :4] - 4 * FI @ Cc).max() < 1e-11
    assert np.abs(r["G"][:, 4:]).max() == 0.0


def test_rotation_invariances(nao48):
    s = nao48
    base = O.system_energy_grad(s)
    rng = np.random.default_rng(3)
    c = s.ncore
    # core-core rotation
    U = np.eye(s.nmo)
    U[:c, :c] = sl.expm((lambda x: x - x.T)(rng.standard_normal((c, c))))
    e1 = O.energy_grad(s.Bp, s.nao, s.h, s.C @ U, c, s.dm1s, s.dm2, with_grad=False)["E"]
    assert abs(e1 - base["E"]) < 1e-11 * abs(base["E"])
    # rotation inside one fragment, RDMs co-rotated: phi'_p = sum_a phi_a V_ap, gamma' = V^T gamma V
    m = s.nact[0]
    V = sl.expm((lambda x: x - x.T)(rng.standard_normal((m, m))))
    U = np.eye(s.nmo)
    U[c:c + m, c:c + m] = V
    d1 = [np.einsum("ap,bq,sab->spq", V, V, s.dm1s[0])] + s.dm1s[1:]
    d2 = [np.einsum("ap,bq,cr,ds,abcd->pqrs", V, V, V, V, s.dm2[0])] + s.dm2[1:]
    e2 = O.energy_grad(s.Bp, s.nao, s.h, s.C @ U, c, d1, d2, with_grad=False)["E"]
    assert abs(e2 - base["E"]) < 1e-11 * abs(base["E"])
    g = base["gorb"]
    o = s.nocc
    assert np.abs(g[:c, :c]).max() < 1e-11 * np.abs(g).max()
    assert np.abs(g[o:, o:]).max() == 0.0
    assert np.abs(g + g.T).max() == 0.0


def test_positivity(nao48):
    s = nao48
    r = O.system_energy_grad(s, with_grad=False)
    Dc = 2 * s.C[:, :s.ncore] @ s.C[:, :s.ncore].T
    assert np.sum(Dc * r["J"]) >= 0
    assert np.sum(Dc * r["K"]) >= 0
    b = O.unpack_block(s.Bp, s.nao)
    v = np.einsum("Pmn,mn->P", b, Dc)
    assert abs(np.sum(Dc * r["J"]) - np.sum(v * v)) < 1e-10 * np.sum(v * v)


def _fd_check(s, ndir, eps=1e-4, seed=0):
    r = O.system_energy_grad(s)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(ndir):
        X = rng.standard_normal((s.nmo, s.nmo))
        X = X - X.T
        X /= np.linalg.norm(X)
        ep = O.energy_grad(s.Bp, s.nao, s.h, s.C @ sl.expm(eps * X), s.ncore, s.dm1s, s.dm2,
                           with_grad=False)["E"]
        em = O.energy_grad(s.Bp, s.nao, s.h, s.C @ sl.expm(-eps * X), s.ncore, s.dm1s, s.dm2,
                           with_grad=False)["E"]
        an = float(np.sum((s.C.T @ r["G"]) * X))
        worst = max(worst, abs((ep - em) / (2 * eps) - an) / max(1.0, abs(an)))
    return worst


def test_finite_differences(nao48):
    assert _fd_check(nao48, 20) < 1e-6


def test_finite_differences_odd_fragment(small3):
    assert _fd_check(small3, 6) < 1e-6


def test_planted_mistakes(nao48, monkeypatch):
    """Each planted slip in the oracle must be caught by one of the pins above."""
    s = nao48
    good = O.system_energy_grad(s, with_grad=False)["E"]
    esc = O.energy_slater_condon(s)
    assert abs(good - esc) < 1e-10

    # (1) wrong sign of the inter-fragment exchange block
    orig = O.active_rdms

    def bad_rdms(d1, d2):
        D, G = orig(d1, d2)
        m = d1[0].shape[-1]
        G2 = G.copy()
        G2[:m, m:, m:, :m] *= -1.0
        G2[m:, :m, :m, m:] *= -1.0
        return D, G2

    monkeypatch.setattr(O, "active_rdms", bad_rdms)
    assert abs(O.system_energy_grad(s, with_grad=False)["E"] - esc) > 1e-6
    monkeypatch.setattr(O, "active_rdms", orig)

    # (2) exchange of the core density without the factor 1/2
    orig_jk = O.df_jk

    def bad_jk(Bp, n, dms, l0=0, l1=None):
        J, K = orig_jk(Bp, n, dms, l0, l1)
        return J, [2 * k for k in K]

    monkeypatch.setattr(O, "df_jk", bad_jk)
    assert abs(O.system_energy_grad(s, with_grad=False)["E"] - esc) > 1e-6
    monkeypatch.setattr(O, "df_jk", orig_jk)

    # (3) a transposed C in the half transform of Eq. ao2mo_1
    orig_ao = O.ao2mo_active

    def bad_ao(Bp, n, C_a, l0=0, l1=None):
        Ct = np.ascontiguousarray(np.roll(C_a, 1, axis=0))
        return orig_ao(Bp, n, Ct, l0, l1)

    monkeypatch.setattr(O, "ao2mo_active", bad_ao)
    assert abs(O.system_energy_grad(s, with_grad=False)["E"] - esc) > 1e-6
    monkeypatch.setattr(O, "ao2mo_active", orig_ao)

    # (4) a dropped factor 2 in the active gradient columns must fail the FD pin
    orig_eg = O.energy_grad

    def bad_grad(*a, **k):
        r = orig_eg(*a, **k)
        if "G" in r:
            c = a[4]
            na = sum(d.shape[-1] for d in a[5])
            r["G"][:, c:c + na] *= 0.5
        return r

    monkeypatch.setattr(O, "energy_grad", bad_grad)
    assert _fd_check(s, 3) > 1e-3
    monkeypatch.setattr(O, "energy_grad", orig_eg)

    # (5) the packed triangle unpacked in the upper triangle's row order: both unpacking pins
    # must fail (every energy route unpacks through the same function, so they cannot see it)
    orig_up = O.unpack_block

    def bad_unpack(Bp_rows, n):
        out = np.zeros((Bp_rows.shape[0], n, n))
        mu, nu = np.triu_indices(n)
        out[:, mu, nu] = Bp_rows
        out[:, nu, mu] = Bp_rows
        return out

    monkeypatch.setattr(O, "unpack_block", bad_unpack)
    with pytest.raises(AssertionError):
        test_unpack_block_packed_index_convention()
    with pytest.raises(AssertionError):
        test_unpacked_generator_band(s)
    monkeypatch.setattr(O, "unpack_block", orig_up)


@pytest.fixture(scope="module")
def many_blocks():
    # 517 auxiliary rows: the oracle's blocks along P (at most 240, the paper's N_blk) are
    # 240 + 240 + 37, so every blocked sum crosses two block edges and ends on a ragged block
    return make_system(11, 517, 2, [(2, 2), (2, 3)], seed=2024)


def test_blocking_over_P(many_blocks):
    """The blocked Tier B sums against unblocked definitions, with several blocks along P."""
    s = many_blocks
    n = s.nao
    assert O.block_size(n, s.naux) == 240 and s.naux % 240 != 0
    r = O.system_energy_grad(s)
    # energy: Tier A builds (pq|rs) from all of B at once
    ea = O.energy_tier_a(s.Bp, n, s.h, s.C, s.ncore, s.dm1s, s.dm2)
    assert abs(r["E"] - ea) < 1e-12 * abs(ea)
    # J and K against the 4-index integrals
    eri = O.ao_eri(s.Bp, n)
    rng = np.random.default_rng(3)
    D = rng.standard_normal((n, n))
    D = D + D.T
    (J,), (K,) = O.df_jk(s.Bp, n, [D])
    assert np.abs(J - np.einsum("mnls,ls->mn", eri, D)).max() < 1e-11
    assert np.abs(K - np.einsum("mlsn,ls->mn", eri, D)).max() < 1e-11
    # active integrals against the unblocked MO transform
    a = s.nactive
    C_a = s.C[:, s.ncore:s.ncore + a]
    e_act, _ = O.ao2mo_active(s.Bp, n, C_a)
    assert np.abs(e_act - O.mo_eri(s.Bp, n, C_a)).max() < 1e-12 * np.abs(e_act).max()
    # gradient: central differences
    assert _fd_check(s, 4) < 1e-6
    # slices of the auxiliary index that start and end inside blocks add up to the whole
    # (the one-electron matrix in one slice only)
    parts = [(0, 100, s.h), (100, 250, 0 * s.h), (250, 517, 0 * s.h)]
    tot_E, tot_G = 0.0, 0.0
    for l0, l1, h in parts:
        p = O.energy_grad(s.Bp, n, h, s.C, s.ncore, s.dm1s, s.dm2, l0=l0, l1=l1)
        tot_E += p["E"]
        tot_G = tot_G + p["G"]
    assert abs(tot_E - r["E"]) < 1e-12 * abs(r["E"])
    assert np.abs(tot_G - r["G"]).max() < 1e-12 * np.abs(r["G"]).max()


def test_planted_dropped_ragged_block(many_blocks, monkeypatch):
    """A blocked loop that drops its last, ragged block must fail the pin above."""
    s = many_blocks
    ea = O.energy_tier_a(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2)
    orig = O.p_blocks

    def bad_blocks(Bp, n, l0=0, l1=None, nblk=240):
        for a, b, blk in orig(Bp, n, l0, l1, nblk):
            if b - a == 240:
                yield a, b, blk

    monkeypatch.setattr(O, "p_blocks", bad_blocks)
    assert abs(O.system_energy_grad(s, with_grad=False)["E"] - ea) > 1e-6 * abs(ea)


SWEEP = [
    # (nao, naux, ncore, fragments (nelec, norb), nmo, seed)
    (9, 27, 0, [(2, 3)], None, 101),                     # no core, one open fragment
    (10, 33, 4, [(1, 2), (3, 3)], None, 102),            # two odd-electron fragments
    (12, 41, 1, [(2, 2), (2, 2), (2, 2)], 10, 103),      # three fragments, nmo < nao
    (11, 250, 3, [(4, 3)], None, 104),                   # fragment with a hole pair; 2 blocks
    (13, 29, 2, [(0, 2), (4, 4)], 12, 105),              # an empty fragment (no electrons)
    (8, 20, 3, [], None, 106),                           # closed shell only
]


@pytest.mark.parametrize("nao,naux,ncore,frags,nmo,seed", SWEEP)
def test_energy_three_ways_sweep(nao, naux, ncore, frags, nmo, seed):
    """Tier B (J/K form), Tier A (explicit MO integrals, full-molecule RDMs) and Slater-Condon
    over the explicit product CI vector agree on systems of varied shape, and the analytic
    gradient matches central differences there."""
    s = make_system(nao, naux, ncore, frags, seed=seed, nmo=nmo)
    eb = O.system_energy_grad(s, with_grad=False)["E"]
    ea = O.energy_tier_a(s.Bp, s.nao, s.h, s.C, s.ncore, s.dm1s, s.dm2)
    esc = O.energy_slater_condon(s)
    assert abs(ea - eb) < 1e-12 * max(1.0, abs(eb))
    assert abs(esc - eb) < 1e-12 * max(1.0, abs(eb))
    assert _fd_check(s, 3, seed=seed) < 1e-6
