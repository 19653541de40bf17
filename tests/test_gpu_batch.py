"""Batched solve of uneven instances: every result equals the single-instance solve and the oracle."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for

pytestmark = pytest.mark.gpu

SHAPES = [(4, 9, 51), (3, 12, 52), (5, 20, 53), (6, 30, 0), (4, 40, 54), (2, 7, 55)]


@pytest.mark.parametrize("precision,concurrency", [(0, 3), (1, 2)])
def test_batch_matches_single_solves(precision, concurrency):
    from paper_2003_12923_gb300 import esmp2
    insts = [synth.make_instance(No, Nv, s) for (No, Nv, s) in SHAPES]
    st, res = esmp2.batch_solve(insts, tol=1e-11, maxit=3000, precision=precision, concurrency=concurrency)
    assert st == esmp2.OK, [r["message"] for r in res]
    for inst, r in zip(insts, res):
        h = handle_for(inst)
        h.solve(tol=1e-11, maxit=3000)
        e = h.energy()
        assert r["status"] == esmp2.OK and r["rel_residual"] <= 1e-11
        assert abs(r["E2"] - e["E2"]) < 1e-10, (r["E2"], e["E2"])
        assert r["kernel_launches"] > 0
    ref = o2.solve(top.prepare(insts[0]), tol=1e-12)
    assert abs(res[0]["E2"] - ref["E2"]) < 1e-10


def test_batch_reports_per_instance_errors():
    from paper_2003_12923_gb300 import esmp2
    good = synth.make_instance(3, 8, 61)
    bad = dict(synth.make_instance(3, 8, 62))
    bad["F"] = bad["F"].copy()
    bad["F"][1, 2] += 1.0   # not symmetric
    st, res = esmp2.batch_solve([good, bad, good], tol=1e-10, concurrency=2)
    assert st == esmp2.ERR_INVALID_ARG
    assert [r["status"] for r in res] == [esmp2.OK, esmp2.ERR_INVALID_ARG, esmp2.OK]
    assert "symmetric" in res[1]["message"]
