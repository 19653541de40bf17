"""Pins of O1 (the determinant-space definition) against textbook identities, closed
forms and invariants -- none of them re-derives O1's own formulas."""
import itertools

import numpy as np
import pytest

import synth
from oracle import jw, top


def _inst(No, Nv, seed, **kw):
    return synth.make_instance(No, Nv, seed, full_eri=True, **kw)


def test_anticommutation():
    # {a_p, a_q^+} = delta_pq and {a_p, a_q} = 0 on the whole Fock space of 8 spin orbitals
    sys = jw.System(2, 2)
    nso = 2 * sys.N
    n = 1 << nso

    def op(fn, k):
        M = np.zeros((n, n))
        for d in range(n):
            sg, dd = fn(d, k)
            if sg:
                M[dd, d] = sg
        return M

    a = [op(jw.ann, k) for k in range(nso)]
    c = [op(jw.cre, k) for k in range(nso)]
    for p in range(nso):
        assert np.array_equal(c[p], a[p].T)
        for q in range(nso):
            assert np.array_equal(a[p] @ c[q] + c[q] @ a[p], np.eye(n) * (p == q))
            assert not np.any(a[p] @ a[q] + a[q] @ a[p])


def _chain(det, ops):
    sign = 1
    for kind, k in ops:
        sg, det = (jw.ann if kind == "a" else jw.cre)(det, k)
        if sg == 0:
            return 0, 0
        sign *= sg
    return sign, det


def _h_and_eri(No, Nv, seed):
    inst = _inst(No, Nv, seed)
    rng = np.random.default_rng(seed)
    N = No + Nv
    h = rng.standard_normal((N, N)) * 0.3
    h = h + h.T
    return h, inst["eri"]


def test_reference_energy_textbook():
    # <Phi|H|Phi> = sum_i 2 h_ii + sum_ij [2 (ii|jj) - (ij|ji)]  (closed-shell determinant)
    No, Nv = 2, 3
    h, g = _h_and_eri(No, Nv, 3)
    sys = jw.System(No, Nv)
    phi = {sys.phi: 1.0}
    e = jw.dot(phi, jw.apply_hamiltonian(sys, phi, h, g))
    ref = sum(2 * h[i, i] for i in range(No)) + sum(2 * g[i, i, j, j] - g[i, j, j, i]
                                                    for i in range(No) for j in range(No))
    assert abs(e - ref) < 1e-12


def test_single_and_double_matrix_elements_textbook():
    No, Nv = 2, 3
    h, g = _h_and_eri(No, Nv, 5)
    sys = jw.System(No, Nv)
    Hphi = jw.apply_hamiltonian(sys, {sys.phi: 1.0}, h, g)
    for i in range(No):
        for a in range(No, No + Nv):
            # Brillouin / Slater-Condon: <Phi_i^a|H|Phi> = f_ai, f = h + sum_j [2(ai|jj) - (aj|ji)]
            f = h[a, i] + sum(2 * g[a, i, j, j] - g[a, j, j, i] for j in range(No))
            sg, d = sys.excite([(i, 0)], [(a, 0)])
            assert abs(sg * Hphi.get(d, 0.0) - f) < 1e-12
    for (i, j) in itertools.product(range(No), repeat=2):
        for (a, b) in itertools.product(range(No, No + Nv), repeat=2):
            # opposite spin: <ab||ij> = (ai|bj); same spin: (ai|bj) - (aj|bi)
            sg, d = sys.excite([(i, 0), (j, 1)], [(a, 0), (b, 1)])
            assert abs(sg * Hphi.get(d, 0.0) - g[a, i, b, j]) < 1e-12
            if i < j and a < b:
                sg, d = sys.excite([(i, 0), (j, 0)], [(a, 0), (b, 0)])
                assert abs(sg * Hphi.get(d, 0.0) - (g[a, i, b, j] - g[a, j, b, i])) < 1e-12


def test_top_basis_and_reference_state():
    No, Nv = 3, 4
    inst = _inst(No, Nv, 11)
    C = top.normalise_singles(inst["C"])
    U, lam, Wv = top.top_basis(C)
    assert np.allclose(U.T @ U, np.eye(No), atol=1e-13)
    assert np.allclose(Wv.T @ Wv, np.eye(Nv), atol=1e-13)
    assert np.allclose(U.T @ C @ Wv[:, :No], np.diag(lam), atol=1e-13)
    assert np.all(np.diff(lam) <= 0)
    r = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    assert abs(jw.dot(r.psi0, r.psi0) - 1.0) < 1e-13
    # gamma is diagonal in the TOP basis: 2 - 2 lam^2 on u, 2 lam^2 on u', 0 on the AVOs
    g = np.zeros(No + Nv)
    g[:No] = 2 - 2 * lam ** 2
    g[No:2 * No] = 2 * lam ** 2
    assert np.allclose(r.gamma, np.diag(g), atol=1e-13)
    assert abs(r.E0 - float(np.sum(g * np.diag(r.F_top)))) < 1e-12
    # the same state expressed in the ESMF basis (Eq. psi0) has the same energies
    sys = r.sys
    psi_orig = jw.psi0_from_singles(sys, C)
    gamma_o = jw.density(sys, psi_orig)
    h_o = inst["F"] - jw.two_electron_fock(gamma_o, inst["eri"])
    e_orig = jw.dot(psi_orig, jw.apply_hamiltonian(sys, psi_orig, h_o, inst["eri"]))
    e_top = jw.dot(r.psi0, jw.apply_hamiltonian(sys, r.psi0, r.h, r.eri_top))
    assert abs(e_orig - e_top) < 1e-11
    assert abs(jw.dot(psi_orig, jw.apply_one_body(sys, psi_orig, inst["F"])) - r.E0) < 1e-12


def test_n_space_rhs_vanishes_and_operator_symmetric():
    # Eq. triples_element: <T|H|Psi0> = 0 unless the triple holds a transition-orbital pair
    No, Nv = 3, 4
    inst = _inst(No, Nv, 2)
    r = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    for d, cl in r.cls.items():
        if cl == "N":
            assert abs(r.b.get(d, 0.0)) < 1e-15
    assert np.abs(r.A - r.A.T).max() < 1e-14
    assert np.linalg.eigvalsh(r.A).min() > 0


def test_closed_form_diagonal_case():
    # F diagonal and C = [diag(lam) 0]: the TOP basis is the input basis, A is diagonal and
    # E2 = -sum_I b_I^2 / (sum_particles F_pp - sum_holes F_hh - omega).
    No, Nv = 3, 4
    inst = _inst(No, Nv, 8)
    F = np.diag(np.diag(inst["F"]))
    C = np.zeros((No, Nv))
    C[0, 0], C[1, 1], C[2, 2] = 0.9, 0.4, 0.2
    r = jw.solve(F, inst["eri"], C, No, Nv)
    Cn = top.normalise_singles(C)
    lam = np.diag(Cn[:, :No])
    fd = np.diag(F)
    omega = np.sum(2 * lam ** 2 * (fd[No:2 * No] - fd[:No]))
    e2 = 0.0
    for d, bd in r.b.items():
        holes, parts = r.sys.excitation(d)
        den = sum(fd[p] for p, _ in parts) - sum(fd[h] for h, _ in holes) - omega
        e2 -= bd * bd / den
    assert abs(r.E2 - e2) < 1e-14 * max(1.0, abs(e2))


def _fragments(NoA, NvA, NoB, NvB, seed):
    """Two non-interacting fragments: block-diagonal F with zero occupied-virtual block,
    integrals only within a fragment, rank-1 singles on fragment A."""
    No, Nv = NoA + NoB, NvA + NvB
    N = No + Nv
    occA, occB = list(range(NoA)), list(range(NoA, No))
    virA, virB = list(range(No, No + NvA)), list(range(No + NvA, N))
    fragA, fragB = occA + virA, occB + virB
    rng = np.random.default_rng(seed)
    F = np.zeros((N, N))
    for frag, occ, vir in ((fragA, occA, virA), (fragB, occB, virB)):
        for blk in (occ, vir):
            M = rng.standard_normal((len(blk), len(blk))) * 0.05
            F[np.ix_(blk, blk)] = M + M.T
        F[occ, occ] += rng.uniform(-2.0, -0.8, len(occ))
        F[vir, vir] += rng.uniform(0.4, 3.0, len(vir))
    full = synth.eri_block("full", No, Nv, seed, 2e-2)
    eri = np.zeros_like(full)
    for frag in (fragA, fragB):
        ix = np.ix_(frag, frag, frag, frag)
        eri[ix] = full[ix]
    C = np.zeros((No, Nv))
    C[0, 0] = 1.0
    return F, eri, C, (occA, virA, occB, virB)


def _mp2_closed_shell(F, eri, occ, vir):
    eo, Uo = np.linalg.eigh(F[np.ix_(occ, occ)])
    ev, Uv = np.linalg.eigh(F[np.ix_(vir, vir)])
    g = eri[np.ix_(occ, vir, occ, vir)]
    g = np.einsum("iajb,ik,al,jm,bn->klmn", g, Uo, Uv, Uo, Uv)
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(g * (2 * g - g.transpose(0, 3, 2, 1)) / den))


def test_size_intensivity_fragment_mp2():
    # Sec. III.F analogue: adding a non-interacting closed-shell fragment B adds exactly the
    # textbook MP2 energy of B to E2 (so the excitation energy is unchanged).
    NoA, NvA, NoB, NvB = 1, 2, 2, 2
    F, eri, C, (occA, virA, occB, virB) = _fragments(NoA, NvA, NoB, NvB, seed=21)
    No, Nv = NoA + NoB, NvA + NvB
    r = jw.solve(F, eri, C, No, Nv)
    ia = occA + virA
    rA = jw.solve(F[np.ix_(ia, ia)], eri[np.ix_(ia, ia, ia, ia)], C[:NoA, :NvA], NoA, NvA)
    mp2 = _mp2_closed_shell(F, eri, occB, virB)
    assert abs(mp2) > 1e-5
    assert abs((r.E2 - rA.E2) - mp2) < 1e-12


def test_missing_integral_blocks_do_not_matter():
    # b = Q H Psi0 needs only ovov / ooov / ovvv; oooo, vvvv and (oo|vv) may be anything
    No, Nv = 3, 4
    inst = _inst(No, Nv, 13)
    r1 = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    e = inst["eri"].copy()
    o, v = slice(0, No), slice(No, No + Nv)
    rnd = synth.eri_block("full", No, Nv, 99, 5e-2)
    for blk in [(o, o, o, o), (v, v, v, v), (o, o, v, v), (v, v, o, o)]:
        e[blk] = rnd[blk]
    r2 = jw.solve(inst["F"], e, inst["C"], No, Nv)
    assert abs(r1.E2 - r2.E2) < 1e-14


def test_invariance_sign_flip_and_relabel():
    No, Nv = 3, 4
    inst = _inst(No, Nv, 17)
    r1 = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    N = No + Nv
    perm = np.array([2, 0, 1] + list(range(No, N))[::-1])
    D = np.diag([1, -1, 1, -1, 1, 1, -1.0])
    T = D[:, perm]          # new orbital k = sign * old orbital perm[k]
    F2 = T.T @ inst["F"] @ T
    e2 = np.einsum("pqrs,pi,qj,rk,sl->ijkl", inst["eri"], T, T, T, T)
    C2 = T[:No, :No].T @ inst["C"] @ T[No:, No:]
    r2 = jw.solve(F2, e2, C2, No, Nv)
    assert abs(r1.E2 - r2.E2) < 1e-13


def test_eta_extremes():
    # eta above the largest singular value: L is empty and every triple is diagonal.
    No, Nv = 3, 4
    inst = _inst(No, Nv, 19)
    r = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv, eta=10.0)
    assert not any(c == "L" for c in r.cls.values())
    # eta = 0: every transition-pair triple is L, S is empty
    r0 = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv, eta=0.0)
    assert not any(c == "S" for c in r0.cls.values())
    r1 = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    assert len({r.E2, r0.E2, r1.E2}) == 3
