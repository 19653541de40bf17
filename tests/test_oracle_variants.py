"""The paper's original (N^7) zeroth-order Hamiltonian and the level shift, in the oracle.

* Eq. old_H0 applies the full Fock operator on every first-order determinant; Eq.
  qfq_replacement keeps it on D + L only and takes its diagonal on S + N.  For a Fock matrix
  that is diagonal in the transition-orbital basis the two coincide (the diagonal part is the
  whole operator); in general they differ, and the parent operator stays positive definite.
* A level shift s adds s to H0 on the first-order space (the intruder-state remedy the paper
  cites for CASPT2): for a diagonal operator E2(s) = -sum_I b_I^2 / (D_I + s) in closed form,
  in general E2(s) = -b.(A + s)^-1 b increases monotonically with s; O2 with a shift equals O1
  with the same shift.
"""
import numpy as np
import pytest

import synth
from oracle import jw, o2, top
from tests.test_oracle_pins import _diagonal_system


def test_original_h0_equals_modified_for_diagonal_fock():
    No, Nv, F, C, eri, _ = _diagonal_system(8)
    r_mod = jw.solve(F, eri, C, No, Nv)
    r_org = jw.solve(F, eri, C, No, Nv, h0="original")
    assert len(r_org.DL) > len(r_mod.DL)            # every triple is iterated in the parent
    assert abs(r_org.E2 - r_mod.E2) < 1e-14 * max(1.0, abs(r_mod.E2))


def test_original_h0_differs_in_general_and_is_positive_definite():
    No, Nv = 3, 4
    inst = synth.make_instance(No, Nv, 19, sigma_off=3e-2, full_eri=True)
    r_mod = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    r_org = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv, h0="original")
    assert np.linalg.eigvalsh(r_org.A).min() > 0
    assert np.abs(r_org.A - r_org.A.T).max() < 1e-14
    assert abs(r_org.E2 - r_mod.E2) > 1e-8
    # the doubles block of the parent operator is the modified one's (both apply full F on D)
    nd = [k for k, d in enumerate(r_org.DL) if r_org.cls[d] == "D"]
    nd_m = [k for k, d in enumerate(r_mod.DL) if r_mod.cls[d] == "D"]
    assert [r_org.DL[k] for k in nd] == [r_mod.DL[k] for k in nd_m]
    assert np.abs(r_org.A[np.ix_(nd, nd)] - r_mod.A[np.ix_(nd_m, nd_m)]).max() == 0.0


@pytest.mark.parametrize("h0", ["modified", "original"])
def test_level_shift_closed_form_for_diagonal_operator(h0):
    No, Nv, F, C, eri, _ = _diagonal_system(8)
    r0 = jw.solve(F, eri, C, No, Nv, h0=h0)
    for s in (0.05, 0.4):
        rs = jw.solve(F, eri, C, No, Nv, h0=h0, shift=s)
        closed = -sum(bd * bd / (r0.diag_energy(d) + s) for d, bd in r0.b.items())
        assert abs(rs.E2 - closed) < 1e-13 * max(1.0, abs(closed))


def test_level_shift_monotonic_and_o2_matches_o1():
    No, Nv = 3, 5
    inst = synth.make_instance(No, Nv, 2, full_eri=True, sigma_off=0.05)
    prep = top.prepare(inst)
    e_prev = None
    for s in (0.0, 0.1, 0.5):
        r = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv, shift=s)
        res = o2.solve(prep, tol=1e-12, shift=s)
        assert abs(res["E2"] - r.E2) < 1e-13
        assert abs(res["E2_S"] - r.parts["S"]) < 1e-14
        if e_prev is not None:
            assert r.E2 > e_prev
        e_prev = r.E2
    assert e_prev < 0
