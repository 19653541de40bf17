"""Host-side checks of the inputs the GPU failure-path tests use: the intruder-state instance
has an operator that is not positive definite (O1, explicit matrix: every eigenvalue is
negative) and the oracle's CG stops on a non-positive curvature p.Ap (Sec. III.A solves by
CG, which needs a positive definite operator)."""
import numpy as np
import pytest

import synth
from oracle import jw, o2, top
from tests.gpu_util import indefinite_instance


def test_indefinite_instance_has_negative_curvature():
    inst = indefinite_instance(2, 4, 5)
    full = synth.eri_block("full", 2, 4, 5)
    r = jw.solve(inst["F"], full, inst["C"], 2, 4)
    ev = np.linalg.eigvalsh(r.A)
    assert ev.max() < 0


@pytest.mark.parametrize("No,Nv", [(3, 6), (4, 12)])
def test_oracle_cg_reports_indefinite(No, Nv):
    inst = indefinite_instance(No, Nv, 5)
    with pytest.raises(RuntimeError, match="positive definite"):
        o2.solve(top.prepare(inst), tol=1e-10)
