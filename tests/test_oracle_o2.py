"""Pins of O2 (amplitude-level oracle): agreement with the determinant-space definition O1
on random tiny systems, operator symmetry, element sampling, and the fragment MP2 limit at
sizes O1 cannot reach."""
import numpy as np
import pytest

import synth
from oracle import jw, o2, top
from tests.test_oracle_jw import _fragments, _mp2_closed_shell


def _blocks_from_det(r, st):
    b = jw.state_to_blocks(r.sys, st)
    return np.stack([b[k] for k in jw.BLOCKS])


def _prep_from(F, eri, C, No, Nv):
    inst = {"No": No, "Nv": Nv, "F": F, "C": C, "ovov": eri[:No, No:, :No, No:].copy(),
            "ooov": eri[:No, :No, :No, No:].copy(), "ovvv": eri[:No, No:, No:, No:].copy()}
    return top.prepare(inst)


@pytest.mark.parametrize("No,Nv,seed", [(3, 4, 1), (3, 5, 2), (4, 5, 3), (3, 6, 4), (4, 4, 5)])
def test_o2_matches_o1(No, Nv, seed):
    inst = synth.make_instance(No, Nv, seed, full_eri=True, sigma_off=0.05)
    r = jw.solve(inst["F"], inst["eri"], inst["C"], No, Nv)
    prep = top.prepare(inst)
    o = o2.O2(prep)
    # omega = E0 - E_Phi[F]: the constant shift of A (E0 = <Psi0|F|Psi0> from O1)
    assert abs(o.omega - (r.E0 - 2 * np.sum(np.diag(r.F_top)[:No]))) < 1e-13
    b = o.rhs()
    bj = _blocks_from_det(r, r.b)
    assert np.abs(b - bj).max() < 1e-14
    rng = np.random.default_rng(seed)
    xb = {k: rng.standard_normal((No, No, Nv, Nv)) for k in jw.BLOCKS}
    st = jw.blocks_to_state(r.sys, xb)
    x = _blocks_from_det(r, st)
    y = o.sigma(x)
    yj = _blocks_from_det(r, jw.apply_A(r, st))
    assert np.abs(y - yj).max() < 1e-12 * max(1.0, np.abs(yj).max())
    res = o2.solve(prep, tol=1e-12)
    assert abs(res["E2"] - r.E2) < 1e-13
    assert abs(res["E2_S"] - r.parts["S"]) < 1e-14
    assert abs(res["E2_D"] - r.parts["D"]) < 1e-13
    assert abs(res["E2_L"] - r.parts["L"]) < 1e-13


def test_o2_operator_symmetric_and_sampling():
    No, Nv = 5, 9
    inst = synth.make_instance(No, Nv, 6)
    prep = top.prepare(inst)
    o = o2.O2(prep)
    rng = np.random.default_rng(0)
    # random vectors in the valid, antisymmetric, spin-consistent subspace: project via A's image
    x = o.sigma(o.rhs() + 0.01 * o.sigma(o.rhs()))
    y = o.sigma(o.rhs())
    assert abs(o2.wdot(x, o.sigma(y)) - o2.wdot(y, o.sigma(x))) < 1e-13 * abs(o2.wdot(x, o.sigma(y)))
    full = o.sigma(x).ravel()
    flat = rng.integers(0, full.size, 500)
    assert np.array_equal(o.sigma_at(x.ravel(), flat), full[flat])
    bfull = o.rhs().ravel()
    assert np.array_equal(o.rhs_at(flat), bfull[flat])


def test_o2_fragment_mp2_limit():
    NoA, NvA, NoB, NvB = 2, 3, 3, 5
    F, eri, C, (occA, virA, occB, virB) = _fragments(NoA, NvA, NoB, NvB, seed=31)
    No, Nv = NoA + NoB, NvA + NvB
    e_ab = o2.solve(_prep_from(F, eri, C, No, Nv), tol=1e-13)["E2"]
    ia = occA + virA
    e_a = o2.solve(_prep_from(F[np.ix_(ia, ia)], eri[np.ix_(ia, ia, ia, ia)], C[:NoA, :NvA], NoA, NvA),
                   tol=1e-13)["E2"]
    mp2 = _mp2_closed_shell(F, eri, occB, virB)
    assert abs((e_ab - e_a) - mp2) < 1e-12


def test_o2_s_space_count():
    # closed-form size of the S space for TOP(1), counted over both spin sectors
    from math import comb
    No, Nv = 4, 7
    inst = synth.make_instance(No, Nv, 3)
    o = o2.O2(top.prepare(inst))
    _, n = o.e2_s()
    r = jw.solve(*(synth.make_instance(No, Nv, 3, full_eri=True)[k] for k in ("F", "eri", "C")), No, Nv)
    assert n == sum(1 for c in r.cls.values() if c == "S")
