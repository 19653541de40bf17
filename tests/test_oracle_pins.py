"""Further pins of the oracle against what the mathematics fixes:

* the AVO completion (Sec. II.A: any completion of V; this build's reading is the Householder
  completion) equals LAPACK's Householder QR (numpy.linalg.qr, mode="complete"), which uses
  the same reflectors and the same sign rule alpha = -sign(x_0) |x|;
* the finite-difference integral derivative equals the closed-form derivative of a system
  whose operator is diagonal (E2 = -sum_I b_I^2 / D_I with b linear in the integrals);
* the derivatives taken from the first-order equation at the oracle's solution equal central
  finite differences of re-solved energies;
* with eta above every singular value (Sec. II.C partition) the L space is empty and E2 is the
  doubles-only solve plus the diagonal triples sum; the doubles part is evaluated
  independently in the semicanonical basis, where the doubles block of H0 is diagonal.
"""
import numpy as np
import pytest

import synth
from oracle import grad, jw, o2, top


@pytest.mark.parametrize("No,Nv,seed", [(1, 4, 1), (3, 7, 2), (5, 11, 3), (6, 30, 4)])
def test_householder_completion_is_lapack_qr(No, Nv, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((Nv, No)))
    Q = top.householder_completion(V)
    Qref, _ = np.linalg.qr(V, mode="complete")
    assert np.abs(Q - Qref).max() < 1e-13
    # the completed basis is orthonormal and its first No columns span V
    assert np.abs(Q.T @ Q - np.eye(Nv)).max() < 1e-13
    assert np.abs(Q[:, :No] @ (Q[:, :No].T @ V) - V).max() < 1e-13


def _diagonal_system(seed):
    No, Nv = 3, 5
    inst = synth.make_instance(No, Nv, seed, full_eri=True)
    F = np.diag([-0.5, -1.0, -1.5, 0.3, 1.0, 1.5, 2.0, 2.5])
    C = np.zeros((No, Nv))
    C[0, 0], C[1, 1], C[2, 2] = 0.9, 0.3, 0.1
    eri = inst["eri"]
    o2inst = {"No": No, "Nv": Nv, "F": F, "C": C, "ovov": eri[:No, No:, :No, No:].copy(),
              "ooov": eri[:No, :No, :No, No:].copy(), "ovvv": eri[:No, No:, No:, No:].copy()}
    return No, Nv, F, C, eri, o2inst


def _images(eri, p, q, r, s, v):
    """Add v to (pq|rs) and every image under the 8-fold permutational symmetry."""
    for (a, b, c, d) in {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}:
        eri[a, b, c, d] += v


@pytest.mark.parametrize("i,a,j,b", [(0, 0, 1, 2), (1, 3, 2, 4), (2, 1, 2, 1), (0, 2, 0, 4)])
def test_fd_ovov_matches_closed_form_diagonal_derivative(i, a, j, b):
    No, Nv, F, C, eri, o2inst = _diagonal_system(8)
    r1 = jw.solve(F, eri, C, No, Nv)
    e2 = eri.copy()
    _images(e2, i, No + a, j, No + b, 1.0)
    r2 = jw.solve(F, e2, C, No, Nv)
    # diagonal operator: E2 = -sum_I b_I^2 / D_I, b affine in the integrals, D independent
    closed = 0.0
    for d, bd in r1.b.items():
        closed -= 2.0 * bd * (r2.b.get(d, 0.0) - bd) / r1.diag_energy(d)
    fd = grad.fd_ovov(o2inst, i, a, j, b, h=1e-5)
    assert abs(closed) > 1e-6
    assert abs(fd - closed) < 1e-8 * max(1.0, abs(closed))


def test_analytic_derivatives_match_finite_differences():
    inst = synth.make_instance(3, 6, 31, sigma_off=2e-2)
    prep = top.prepare(inst)
    x = o2.solve(prep, tol=1e-13)["x"]
    for (p, q) in [(0, 0), (1, 2), (0, 4), (2, 7), (3, 3), (5, 8)]:
        an = grad.analytic_F(inst, x, p, q, prep=prep)
        fd = grad.fd_F(inst, p, q, h=1e-5)
        assert abs(an - fd) < 1e-7 * max(1e-3, abs(fd)), (p, q, an, fd)
    for (i, a, j, b) in [(0, 0, 1, 2), (1, 3, 2, 5), (2, 1, 2, 1), (0, 4, 0, 2)]:
        an = grad.analytic_ovov(inst, x, i, a, j, b, prep=prep)
        fd = grad.fd_ovov(inst, i, a, j, b, h=1e-5)
        assert abs(an - fd) < 1e-7 * max(1e-3, abs(fd)), (i, a, j, b, an, fd)


def test_eta_above_all_singular_values_is_doubles_solve_plus_diagonal_triples():
    No, Nv = 3, 4
    inst = synth.make_instance(No, Nv, 19, sigma_off=3e-2, full_eri=True)
    F, eri, C = inst["F"], inst["eri"], inst["C"]
    r = jw.solve(F, eri, C, No, Nv, eta=10.0)
    assert r.parts["L"] == 0.0
    # triples: every one on the diagonal of F in the TOP basis
    trip = 0.0
    for d, bd in r.b.items():
        if len(r.sys.excitation(d)[0]) == 3:
            trip -= bd * bd / r.diag_energy(d)
    assert abs((r.parts["S"] + r.parts["N"]) - trip) < 1e-15
    # doubles: the doubles space and Psi0 do not depend on rotations within the occupied and
    # within the virtual orbitals; in the basis that diagonalises F_oo and F_vv the doubles
    # block of (F - E0) is diagonal, so E2_D = -sum_D b_I^2 / (<I|F|I> - E0) there
    _, Uo = np.linalg.eigh(F[:No, :No])
    _, Uv = np.linalg.eigh(F[No:, No:])
    R = np.zeros((No + Nv, No + Nv))
    R[:No, :No], R[No:, No:] = Uo, Uv
    Fs = R.T @ F @ R
    es = top.transform_full_eri(eri, R)
    sysm = jw.System(No, Nv)
    psi0 = jw.psi0_from_singles(sysm, Uo.T @ top.normalise_singles(C) @ Uv)
    gamma = jw.density(sysm, psi0)
    h = Fs - jw.two_electron_fock(gamma, es)
    Hpsi = jw.apply_hamiltonian(sysm, psi0, h, es)
    E0 = jw.dot(psi0, jw.apply_one_body(sysm, psi0, Fs))
    e2d = 0.0
    for d, bd in Hpsi.items():
        holes, parts = sysm.excitation(d)
        if len(holes) != 2:
            continue
        occ = sum(Fs[p, p] for s in (0, 1) for p in range(No + Nv) if (d >> sysm.so(p, s)) & 1)
        e2d -= bd * bd / (occ - E0)
    assert abs(r.parts["D"] - e2d) < 1e-12 * max(1.0, abs(e2d))
    assert abs(r.E2 - (e2d + trip)) < 1e-12 * max(1.0, abs(r.E2))
