"""The reduced-cost basis (ESMP2_REDUCED_MIXED): occupied orbitals other than t and virtual
orbitals other than t' diagonalise their blocks of F, so the virtual-index terms are
element-wise.  D and L do not change under rotations that fix t and t' (Sec. II.C), so the
operator in that basis is the same operator: its sigma, solution and E2 must equal the oracle's
(which works in the TOP basis) to the precision of the float32 inner solve / the solve
tolerance."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for, masks, random_block_vector

pytestmark = pytest.mark.gpu


def _torch(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 31), (6, 30, 0), (3, 300, 32), (5, 131, 33)])
def test_sigma_reduced_vs_oracle(No, Nv, seed):
    """x rotated into the reduced-cost basis (float64-exact), the float32 inner sigma with the
    virtual-index terms element-wise, y rotated back: float32 accuracy, no bf16 operand."""
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.02)
    h = handle_for(inst)
    x = random_block_vector(No, Nv, seed + 7)
    y = h.sigma(_torch(x), esmp2.REDUCED_MIXED).cpu().numpy()
    ref = o2.O2(top.prepare(inst)).sigma(x)
    rel = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    assert 1e-9 < rel < 2e-5, rel
    assert float(np.abs(y - ref).max()) <= 1e-4 * float(np.abs(ref).max())
    assert not np.any(y[~masks(No, Nv)])


@pytest.mark.parametrize("No,Nv,seed", [(3, 5, 11), (4, 9, 12), (6, 30, 0), (5, 64, 14), (2, 7, 23)])
def test_solve_reduced_matches_oracle(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=2000, precision=esmp2.REDUCED_MIXED)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11 and info["outer"] >= 1
    for k in ("E2", "E2_D", "E2_L", "E2_S"):
        assert abs(e[k] - ref[k]) < 1e-10, (k, e[k], ref[k])
    # the solution comes back in the TOP basis
    x = h.solution().cpu().numpy()
    assert np.abs(x - ref["x"]).max() < 1e-8 * np.abs(ref["x"]).max()
    # the other forms continue from it (basis changes handled by the library)
    info2 = h.solve(tol=1e-11, maxit=50)
    assert info2["iterations"] <= 2
    info3 = h.solve(tol=1e-11, maxit=2000, precision=esmp2.MIXED_BF16)
    assert info3["rel_residual"] <= 1e-11
    assert abs(h.energy()["E2"] - ref["E2"]) < 1e-10


def test_reduced_needs_packed_inner_solve():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(33, 34, 5)
    h = handle_for(inst)
    with pytest.raises(esmp2.Esmp2Error) as ei:
        h.solve(tol=1e-8, maxit=10, precision=esmp2.REDUCED_MIXED)
    assert ei.value.status == esmp2.ERR_UNSUPPORTED


def test_reduced_matches_contraction_form_at_nv400():
    """Nv = 400 (as the benchmark): in the TOP basis F_vv is far from diagonal (W_v mixes the
    virtual orbitals), so the Jacobi eigenvectors take several sweeps; the reduced-cost E2 must
    equal the tensor-core form's and the float64 form's to the mixed tolerance."""
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(6, 400, 41)
    e = {}
    for name, prec, tol in (("fp64", esmp2.FP64, 1e-10), ("bf16", esmp2.MIXED_BF16, 1e-9),
                            ("reduced", esmp2.REDUCED_MIXED, 1e-9)):
        h = handle_for(inst)
        h.solve(tol=tol, maxit=3000, precision=prec)
        e[name] = h.energy()
        h.close()
    for k in ("E2", "E2_D", "E2_L", "E2_S"):
        assert abs(e["reduced"][k] - e["fp64"][k]) < 1e-8, (k, e["reduced"][k], e["fp64"][k])
        assert abs(e["bf16"][k] - e["fp64"][k]) < 1e-8, (k, e["bf16"][k], e["fp64"][k])


@pytest.mark.parametrize("No,Nv,shift", [(3, 6, 2.0), (2, 5, 1.5)])
def test_minres_on_indefinite_operator_against_o1(No, Nv, shift):
    """An operator with eigenvalues of both signs (occupied orbital energies raised into the
    virtual range): CG stops with INDEFINITE, preconditioned MINRES in the reduced-cost basis
    reaches the energy of the explicitly assembled operator's dense solve (O1)."""
    from paper_2003_12923_gb300 import esmp2
    from oracle import jw
    from tests.gpu_util import indefinite_instance
    inst = indefinite_instance(No, Nv, 5, shift=shift)
    ref = jw.solve(inst["F"], synth.eri_block("full", No, Nv, 5), inst["C"], No, Nv)
    ev = np.linalg.eigvalsh(ref.A)
    assert ev.min() < 0 < ev.max()
    h = handle_for(inst)
    with pytest.raises(esmp2.Esmp2Error) as ei:
        h.solve(tol=1e-10, maxit=500, precision=esmp2.FP64)
    assert ei.value.status == esmp2.ERR_INDEFINITE
    h.close()
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=3000, precision=esmp2.REDUCED_MINRES)
    assert info["rel_residual"] <= 1e-11
    assert abs(h.energy()["E2"] - ref.E2) < 1e-10, (h.energy()["E2"], ref.E2)


def test_minres_matches_cg_on_positive_definite_operator():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(5, 64, 14)
    e = {}
    for prec in (esmp2.FP64, esmp2.REDUCED_MINRES):
        h = handle_for(inst)
        info = h.solve(tol=1e-11, maxit=3000, precision=prec)
        assert info["rel_residual"] <= 1e-11
        e[prec] = h.energy()
        h.close()
    for k in ("E2", "E2_D", "E2_L", "E2_S"):
        assert abs(e[esmp2.REDUCED_MINRES][k] - e[esmp2.FP64][k]) < 1e-10
