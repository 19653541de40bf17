"""Options of the problem statement through the C ABI against the oracle: the level shift of H0
(A -> A + s, every S-space denominator + s; the intruder-state remedy the paper cites) for the
float64 and mixed-precision solves, and the selection of the large transition-orbital pair
(Sec. II.C: eta threshold or n_large; this library builds TOP(1))."""
import numpy as np
import pytest

import synth
from oracle import o2, top

pytestmark = pytest.mark.gpu


def _handle(inst, **kw):
    from paper_2003_12923_gb300 import esmp2
    return esmp2.Handle(inst["F"], inst["ovov"], inst["ooov"], inst["ovvv"], inst["C"], **kw)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 12), (6, 30, 0)])
def test_level_shift_against_oracle(No, Nv, seed, prec):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    p = esmp2.FP64 if prec == "fp64" else esmp2.MIXED_BF16
    prep = top.prepare(inst)
    for s in (0.1, 0.5):
        h = _handle(inst, level_shift=s)
        h.solve(tol=1e-11, maxit=2000, precision=p)
        e = h.energy()
        ref = o2.solve(prep, tol=1e-12, shift=s)
        for k in ("E2", "E2_D", "E2_L"):
            assert abs(e[k] - ref[k]) < 1e-10, (s, k, e[k], ref[k])
        assert abs(e["E2_S"] - ref["E2_S"]) < 1e-12
        h.close()


def test_large_pair_selection():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(5, 13, 13)
    lam = top.prepare(inst)["lam"]
    base = _handle(inst)
    base.solve(tol=1e-11, maxit=500)
    e0 = base.energy()["E2"]
    # eta between the largest and the second singular value selects the same single pair
    h = _handle(inst, eta=0.5 * (lam[0] + lam[1]), n_large=0)
    h.solve(tol=1e-11, maxit=500)
    assert h.energy()["E2"] == e0
    with pytest.raises(esmp2.Esmp2Error) as ei:   # two pairs above eta: TOP(2)
        _handle(inst, eta=0.5 * (lam[1] + lam[2]), n_large=0)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED
    with pytest.raises(esmp2.Esmp2Error) as ei:   # no pair above eta
        _handle(inst, eta=2.0 * lam[0], n_large=0)
    assert ei.value.status == esmp2.ERR_INVALID_ARG
    with pytest.raises(esmp2.Esmp2Error) as ei:
        _handle(inst, n_large=2)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED
    with pytest.raises(esmp2.Esmp2Error) as ei:
        _handle(inst, avo_convention=1)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED
