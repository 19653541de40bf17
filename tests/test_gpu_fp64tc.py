"""Float64-accurate virtual-index terms from exact bf16 digit products on the tensor cores
(ESMP2_FP64_TC): the contraction against the float64 GEMMs on inputs of wide dynamic range,
the sigma against the float64 sigma, and solves against the oracle."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import handle_for, random_block_vector

pytestmark = pytest.mark.gpu

# ragged row tiles, two column tiles, Nv not a multiple of 8
SIZES = [(3, 5, 21), (4, 9, 22), (7, 70, 24), (4, 130, 25), (3, 300, 26), (2, 450, 27), (3, 401, 28)]


def _torch(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("No,Nv,seed", SIZES)
def test_virtual_contraction_fp64tc(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.05)
    h = handle_for(inst)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((5, No, No, Nv, Nv))
    x *= 10.0 ** rng.uniform(-8, 3, (5, No, No, 1, 1))     # slices of very different size
    xt = _torch(x)
    y64 = h.virtual_contraction(xt, esmp2.FP64).cpu().numpy()
    ytc = h.virtual_contraction(xt, esmp2.FP64_TC).cpu().numpy()
    Fmax = np.abs(h.top_basis()[3][No:, No:]).max()
    xmax = np.abs(x).max(axis=(3, 4), keepdims=True)
    # ten digit levels: truncation and dropped pairs stay at the float64 rounding level of
    # the largest possible term sum Nv max|x_s| max|F| of each slice
    bound = 2.0 ** -46 * Nv * xmax * Fmax
    err = np.abs(ytc - y64)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.linalg.norm(ytc - y64) <= 1e-13 * np.linalg.norm(y64)
    # against an extended-precision reference on the two largest slices: within a few float64
    # rounding units of the slice's largest element (bf16 operands: ~1e-3, eight levels ~1e-12)
    F = h.top_basis()[3][No:, No:].astype(np.longdouble)
    flat = x.reshape(-1, Nv, Nv)
    for s in np.argsort(-np.abs(flat).max(axis=(1, 2)))[:2]:
        xs = flat[s].astype(np.longdouble)
        ref = xs @ F + F @ xs
        e_tc = float(np.abs(ytc.reshape(-1, Nv, Nv)[s] - ref).max())
        e_64 = float(np.abs(y64.reshape(-1, Nv, Nv)[s] - ref).max())
        scale = float(np.abs(ref).max())
        assert e_tc <= max(16 * e_64, 2.0 ** -45 * scale), (s, e_tc, e_64, scale)


@pytest.mark.parametrize("No,Nv,seed", [(4, 9, 31), (6, 30, 0), (3, 300, 32)])
def test_sigma_fp64tc_vs_fp64(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed, sigma_off=0.02)
    h = handle_for(inst)
    x = _torch(random_block_vector(No, Nv, seed + 7))
    y64 = h.sigma(x, esmp2.FP64)
    ytc = h.sigma(x, esmp2.FP64_TC)
    assert float((ytc - y64).abs().max()) <= 1e-12 * float(y64.abs().max())


@pytest.mark.parametrize("No,Nv,seed", [(3, 5, 11), (4, 9, 12), (6, 30, 0)])
def test_solve_fp64tc_matches_oracle(No, Nv, seed):
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(No, Nv, seed)
    h = handle_for(inst)
    info = h.solve(tol=1e-11, maxit=2000, precision=esmp2.FP64_TC)
    e = h.energy()
    ref = o2.solve(top.prepare(inst), tol=1e-12)
    assert info["rel_residual"] <= 1e-11
    assert abs(e["E2"] - ref["E2"]) < 1e-10


def test_solve_fp64tc_matches_fp64_at_several_tiles():
    from paper_2003_12923_gb300 import esmp2
    inst = synth.make_instance(4, 130, 25)
    h = handle_for(inst)
    h.solve(tol=1e-11, maxit=2000, precision=esmp2.FP64_TC)
    e_tc = h.energy()["E2"]
    h2 = handle_for(inst)
    h2.solve(tol=1e-11, maxit=2000)
    e64 = h2.energy()["E2"]
    assert abs(e_tc - e64) < 1e-10, (e_tc, e64)
