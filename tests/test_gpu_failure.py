"""Failure paths through the C ABI, with no GPU fault: an operator that is not positive
definite (an intruder-state input) makes both solvers stop with ESMP2_ERR_INDEFINITE and the
next handle works; a bounded device wait that runs out (the self-test's producer issues no
copies, so nothing is in flight) is reported as ESMP2_ERR_TIMEOUT and the context stays usable."""
import time

import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for, indefinite_instance

pytestmark = pytest.mark.gpu


def test_indefinite_operator_is_reported_and_next_handle_works():
    from paper_2003_12923_gb300 import esmp2
    h = handle_for(indefinite_instance(4, 12, 5))
    for prec in (esmp2.FP64, esmp2.MIXED_BF16, esmp2.FP64_TC):
        r = h.solve(tol=1e-10, maxit=200, precision=prec, raise_on_error=False)
        assert r["status"] == esmp2.ERR_INDEFINITE, (prec, r)
    h.close()
    inst = synth.make_instance(4, 12, 3)
    h2 = handle_for(inst)
    h2.solve(tol=1e-11, maxit=500)
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert abs(h2.energy()["E2"] - ref["E2"]) < 1e-10


def test_bounded_wait_runs_out_and_is_reported():
    import torch
    from paper_2003_12923_gb300 import esmp2
    torch.cuda.synchronize()
    for wait_ms in (200, 50):
        t0 = time.perf_counter()
        st = esmp2.selftest_bounded_wait(wait_ms)
        dt = time.perf_counter() - t0
        assert st == esmp2.ERR_TIMEOUT, st
        assert dt >= 0.9 * wait_ms * 1e-3, dt
    # the context is intact: the allocation-free contraction and a handle both work next
    Nv, S = 40, 3
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal((S, Nv, Nv))).cuda()
    Fv = torch.from_numpy(rng.standard_normal((Nv, Nv))).cuda()
    Fv = 0.5 * (Fv + Fv.T)
    y = torch.empty_like(x)
    assert esmp2.virtual_contraction_noalloc(x, Fv, y, S, Nv) == esmp2.OK
    torch.cuda.synchronize()
    ref = x @ Fv + Fv @ x
    assert float((y - ref).abs().max()) < 2e-2 * float(ref.abs().max())
    inst = synth.make_instance(3, 7, 9)
    h = handle_for(inst)
    h.solve(tol=1e-11, maxit=300, precision=esmp2.MIXED_BF16)
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert abs(h.energy()["E2"] - ref["E2"]) < 1e-8
