"""Degenerate sizes through the C ABI against the oracle: one occupied orbital (only the t
pair, so no T, X, Y amplitudes and no S-space pair other than t), Nv = No, and the smallest
non-trivial shapes; float64 and mixed-precision solves with the energy parts held to the
bounds of the regular cases."""
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for

pytestmark = pytest.mark.gpu

CASES = [(1, 4, 21), (2, 2, 22), (2, 7, 23), (3, 3, 24)]


@pytest.mark.parametrize("No,Nv,seed", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_sizes(No, Nv, seed, prec):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    p = esmp2.FP64 if prec == "fp64" else esmp2.MIXED_BF16
    info = h.solve(tol=1e-11, maxit=2000, precision=p)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11
    for k in ("E2", "E2_D", "E2_L"):
        assert abs(e[k] - ref[k]) < 1e-10, (k, e[k], ref[k])
    assert abs(e["E2_S"] - ref["E2_S"]) < 1e-12
    h.close()
