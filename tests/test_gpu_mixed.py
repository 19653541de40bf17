"""The bf16 tcgen05 path: the virtual-index contraction against float64 GEMMs within the
bf16 rounding bound, the mixed sigma against the oracle, and the refined solve against the
oracle to float64 tolerances."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for, masks, random_block_vector

pytestmark = pytest.mark.gpu

# Nv < 128, Nv > 128 (several row tiles), Nv > 256 (two column tiles), Nv not a multiple of 8
SIZES = [(3, 5, 21), (4, 9, 22), (5, 13, 23), (7, 70, 24), (6, 30, 0), (4, 130, 25), (3, 300, 26), (2, 450, 27),
         (3, 401, 28)]


def _torch(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bound(h, x_t, F_vv):
    """Elementwise bound of the bf16 error: each product carries <= 2^-8 relative error
    (both operands rounded to 8 significant bits), fp32 accumulation adds far less."""
    import torch
    Fa = torch.from_numpy(np.abs(F_vv)).cuda()
    xa = x_t.abs().reshape(-1, h.Nv, h.Nv)
    b = xa @ Fa + Fa @ xa
    return (2.0 ** -7) * b.reshape(h.shape) + 1e-30


@pytest.mark.parametrize("No,Nv,seed", SIZES)
def test_virtual_contraction_bf16(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.05)
    h = handle_for(inst)
    rng = np.random.default_rng(seed)
    x = _torch(rng.standard_normal((5, No, No, Nv, Nv)))
    y64 = h.virtual_contraction(x, esmp2.FP64)
    y16 = h.virtual_contraction(x, esmp2.MIXED_BF16)
    F = h.top_basis()[3][No:, No:]
    bound = _bound(h, x, F)
    err = (y16 - y64).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    # and it is not trivially passing: the bf16 result differs from fp64 but tracks it closely
    rel = float(err.norm() / y64.norm())
    assert 1e-6 < rel < 1e-2, rel


@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 31), (6, 30, 0), (3, 300, 32)])
def test_sigma_mixed_vs_oracle(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.02)
    h = handle_for(inst)
    x = random_block_vector(No, Nv, seed + 7)
    xt = _torch(x)
    y = h.sigma(xt, esmp2.MIXED_BF16).cpu().numpy()
    ref = o2.O2(top.prepare(inst)).sigma(x)
    # bf16 operands carry 2^-9 relative rounding (the diagonal terms dominate each element),
    # everything else float32: the result is within a few 1e-3 of the operator, not closer
    # than float32 rounding
    rel = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    assert 1e-6 < rel < 4e-3, rel
    assert float(np.abs(y - ref).max()) <= 2e-2 * float(np.abs(ref).max())
    assert not np.any(y[~masks(No, Nv)])
    # the result keeps the symmetries of the amplitudes: exactly in (a, b), to rounding in (i, j)
    # (the occupied rotation back from the working basis mixes slices)
    assert np.array_equal(y[0], -y[0].transpose(0, 1, 3, 2))
    assert float(np.abs(y[0] + y[0].transpose(1, 0, 2, 3)).max()) <= 1e-12 * float(np.abs(y[0]).max())


@pytest.mark.parametrize("No,Nv,seed", [(3, 5, 11), (4, 9, 12), (5, 13, 13), (6, 30, 0)])
def test_solve_mixed_matches_oracle(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11 and info["outer"] >= 1 and info["sigma_lowp"] > 0
    assert abs(e["E2"] - ref["E2"]) < 1e-10
    assert abs(e["E2_S"] - ref["E2_S"]) < 1e-12
    x = h.solution().cpu().numpy()
    assert np.abs(x - ref["x"]).max() < 1e-8 * np.abs(ref["x"]).max()
    # the plain fp64 solve continues from the mixed solution (basis handled by the library)
    info2 = h.solve(tol=1e-11, maxit=50)
    assert info2["iterations"] <= 2


@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 12), (6, 30, 0), (5, 64, 14)])
def test_solve_mixed_graph_replay_matches_oracle(No, Nv, seed):
    """On a non-default stream the inner PCG iteration is captured once and replayed as a
    CUDA graph; the result must not change."""
    import torch
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        t = {k: torch.from_numpy(inst[k]).cuda() for k in ("F", "ovov", "ooov", "ovvv", "C")}
        h = esmp2.Handle(t["F"], t["ovov"], t["ooov"], t["ovvv"], t["C"], stream=st)
        info = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
        e = h.energy()
        # a second solve from zero on the same handle replays the cached graph
        h.set_solution(torch.zeros(h.shape, dtype=torch.float64, device="cuda"))
        info2 = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
        e2 = h.energy()
    st.synchronize()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11 and info2["rel_residual"] <= 1e-11
    assert abs(e["E2"] - ref["E2"]) < 1e-10
    assert abs(e2["E2"] - ref["E2"]) < 1e-10
    plain = handle_for(inst)
    info3 = plain.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
    assert info3["iterations"] == info["iterations"]


@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 31), (6, 30, 0), (3, 300, 32)])
def test_sigma_tf32_vs_oracle(No, Nv, seed):
    """The tf32 inner sigma: operands keep 10 explicit mantissa bits (the low 13 bits of each
    float32 are ignored, a relative error below 2^-10 per operand), so the result is closer
    to the operator than the bf16 form on the same input and no closer than float32 rounding."""
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.02)
    h = handle_for(inst)
    x = random_block_vector(No, Nv, seed + 7)
    xt = _torch(x)
    y32 = h.sigma(xt, esmp2.MIXED_TF32).cpu().numpy()
    y16 = h.sigma(xt, esmp2.MIXED_BF16).cpu().numpy()
    ref = o2.O2(top.prepare(inst)).sigma(x)
    rel32 = float(np.linalg.norm(y32 - ref) / np.linalg.norm(ref))
    rel16 = float(np.linalg.norm(y16 - ref) / np.linalg.norm(ref))
    assert 1e-7 < rel32 < 1.5e-3, rel32
    assert rel32 < 0.5 * rel16, (rel32, rel16)
    assert float(np.abs(y32 - ref).max()) <= 5e-3 * float(np.abs(ref).max())
    assert not np.any(y32[~masks(No, Nv)])
    assert np.array_equal(y32[0], -y32[0].transpose(0, 1, 3, 2))


@pytest.mark.parametrize("No,Nv,seed", [(3, 5, 11), (6, 30, 0), (5, 64, 14)])
def test_solve_tf32_matches_oracle(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_TF32)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11 and info["outer"] >= 1 and info["sigma_lowp"] > 0
    assert abs(e["E2"] - ref["E2"]) < 1e-10
    x = h.solution().cpu().numpy()
    assert np.abs(x - ref["x"]).max() < 1e-8 * np.abs(ref["x"]).max()
    # bf16 and tf32 solves alternate on one handle (separate operands, graph rebuilt)
    import torch
    h.set_solution(torch.zeros(h.shape, dtype=torch.float64, device="cuda"))
    info2 = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
    assert info2["rel_residual"] <= 1e-11
    assert abs(h.energy()["E2"] - ref["E2"]) < 1e-10
    ms = h.profile_sigma(h.rhs(), precision=esmp2.MIXED_TF32, reps=1)
    assert ms[0] >= 0.0 and ms[1] > 0.0 and ms[4] > 0.0


def test_tf32_needs_packed_inner_solve():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(33, 34, 5)
    h = handle_for(inst)
    with pytest.raises(esmp2.Esmp2Error) as ei:
        h.solve(tol=1e-8, maxit=10, precision=esmp2.MIXED_TF32)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED
