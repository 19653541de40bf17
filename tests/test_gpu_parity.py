"""GPU (C ABI) against the oracle, element by element, in float64."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for, masks, random_block_vector, sample_indices

pytestmark = pytest.mark.gpu

# sizes: several GEMM tiles, ragged tails (Nv not a multiple of the tile), odd No
SMALL = [(3, 5, 11), (4, 9, 12), (5, 13, 13), (7, 70, 14), (6, 30, 0)]


def _torch(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("No,Nv,seed", SMALL)
def test_top_basis(No, Nv, seed):
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    U, lam, Wv, F = h.top_basis()
    p = top.prepare(inst)
    assert np.abs(lam - p["lam"]).max() < 1e-13
    assert np.abs(U - p["U"]).max() < 1e-11
    assert np.abs(Wv - p["Wv"]).max() < 1e-11
    assert np.abs(F - p["F"]).max() < 1e-11
    o = o2.O2(p)
    assert abs(h.omega - o.omega) < 1e-12


@pytest.mark.parametrize("No,Nv,seed", SMALL)
def test_rhs(No, Nv, seed):
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    b = h.rhs().cpu().numpy()
    ref = o2.O2(top.prepare(inst)).rhs()
    assert np.abs(b - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("No,Nv,seed", SMALL)
def test_sigma_fp64(No, Nv, seed):
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.02)
    h = handle_for(inst)
    x = random_block_vector(No, Nv, seed + 100, singlet=False)   # the float64 sigma takes any S
    y = h.sigma(_torch(x)).cpu().numpy()
    ref = o2.O2(top.prepare(inst)).sigma(x)
    err = np.abs(y - ref).max()
    assert err < 1e-11 * np.abs(ref).max(), err
    assert not np.any(y[~masks(No, Nv)])


@pytest.mark.parametrize("No,Nv,seed", [(3, 5, 11), (4, 9, 12), (5, 13, 13), (6, 30, 0)])
def test_solve_energy_fp64(No, Nv, seed):
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=500)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11
    assert abs(e["E2"] - ref["E2"]) < 1e-10
    assert abs(e["E2_S"] - ref["E2_S"]) < 1e-12
    assert abs(e["E2_D"] - ref["E2_D"]) < 1e-10
    assert abs(e["E2_L"] - ref["E2_L"]) < 1e-10
    x = h.solution().cpu().numpy()
    assert np.abs(x - ref["x"]).max() < 1e-8 * np.abs(ref["x"]).max()


def test_warm_start_and_errors():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(4, 9, 5)
    h = handle_for(inst)
    with pytest.raises(esmp2.Esmp2Error) as ei:
        h.energy()
    assert ei.value.status == esmp2.ERR_STATE
    r = h.solve(tol=1e-10, maxit=2, raise_on_error=False)
    assert r["status"] == esmp2.ERR_NOT_CONVERGED and r["iterations"] == 2
    r2 = h.solve(tol=1e-10, maxit=500)
    r3 = h.solve(tol=1e-10, maxit=500)  # warm start from the converged solution
    assert r3["iterations"] == 0 and r3["rel_residual"] <= 1e-10
    bad = dict(inst)
    bad["F"] = inst["F"].copy()
    bad["F"][0, 1] = np.nan
    with pytest.raises(esmp2.Esmp2Error) as ei:
        handle_for(bad)
    assert ei.value.status == esmp2.ERR_INVALID_ARG
    with pytest.raises(esmp2.Esmp2Error) as ei:
        esmp2.Handle(inst["F"], inst["ovov"], inst["ooov"], inst["ovvv"], inst["C"], spin=-1)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED
