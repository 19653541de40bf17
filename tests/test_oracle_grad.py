"""Pin of the finite-difference reference gradient: for a diagonal Fock matrix and C = [diag(l) 0]
the operator is diagonal, E2 = -sum_I b_I^2 / D_I with b independent of the diagonal of F, so
dE2/dF_pp = sum_I (b_I / D_I)^2 (n_I(p) - d omega / dF_pp) in closed form (O1 determinant data)."""
import numpy as np

import synth
from oracle import grad, jw, top


def test_fd_matches_closed_form_diagonal_derivative():
    No, Nv = 3, 5
    inst = synth.make_instance(No, Nv, 8, full_eri=True)
    # dominant pair at HOMO/LUMO keeps (H0 - E0) positive definite, so CG applies
    F = np.diag([-0.5, -1.0, -1.5, 0.3, 1.0, 1.5, 2.0, 2.5])
    C = np.zeros((No, Nv))
    C[0, 0], C[1, 1], C[2, 2] = 0.9, 0.3, 0.1
    r = jw.solve(F, inst["eri"], C, No, Nv)
    lam = np.diag(top.normalise_singles(C)[:, :No])
    N = No + Nv
    fd = np.diag(F)
    omega = np.sum(2 * lam ** 2 * (fd[No:2 * No] - fd[:No]))
    dom = np.zeros(N)
    dom[:No] = -2 * lam ** 2
    dom[No:2 * No] = 2 * lam ** 2
    analytic = np.zeros(N)
    for d, bd in r.b.items():
        holes, parts = r.sys.excitation(d)
        D = sum(fd[p] for p, _ in parts) - sum(fd[hh] for hh, _ in holes) - omega
        occ = np.zeros(N)
        for p, _ in parts:
            occ[p] += 1
        for hh, _ in holes:
            occ[hh] -= 1
        analytic += (bd / D) ** 2 * (occ - dom)
    o2inst = {"No": No, "Nv": Nv, "F": F, "C": C, "ovov": inst["eri"][:No, No:, :No, No:].copy(),
              "ooov": inst["eri"][:No, :No, :No, No:].copy(), "ovvv": inst["eri"][:No, No:, No:, No:].copy()}
    for p in range(N):
        assert abs(grad.fd_F(o2inst, p, p, h=1e-5) - analytic[p]) < 1e-8 * max(1.0, abs(analytic[p]))
